// fd_engine_tb.cuh -- temporally blocked variant of the engine (FP32 state and accumulation;
// FP32, BF16 or FP16 history; full, short and adaptive memory).
//
// The full-memory sum is a Toeplitz product: row delta^r enters step k with weight
// psi_{k-r} (eq. frac_norxn), so the steps k = kb .. kb+T-1 of one block all use the same old
// rows.  For block b (kb = bT) this kernel splits each step's sum into
//   far:  rows r <= kb-T-1, read ONCE per block and multiplied into T accumulators with the
//         sliding coefficient window psi_{kb-r} .. psi_{kb+T-1-r};
//   near: the previous block's rows kb-T .. kb-1, one near unit per (block, tile) once block b-1
//         is done (blocks of 16 and more);
//   mid:  with blocks of 32 and 64, the block's own rows of earlier 16-step sub-blocks, one mid
//         unit per (block, sub-block, tile);
//   head: the remaining newest rows (the step's own sub-block or block), summed step by step in
//         the per-tile update.
// Far rows of block b are complete once block b-2 has been updated, so the far streaming of
// block b+1 overlaps the T sequential updates of block b.  History traffic drops by about T
// while the multiply-adds stay the same: the sum is the paper's, only grouped differently.
// Short memory (eq. frac_shortmemory) is the same product with psi_m set to 0 for m > L.
// Adaptive memory (Definitions 3.1-3.2) is the same product with the weights g(m) that the
// medians settle on (psi_m on the base interval, d psi_m at a median, 0 between), for all rows
// above the longest tail of the block's steps; the update units add those few oldest rows with
// each step's own weights, and the CUDA-core far loop skips the zero weights.
// The far product is a contraction: on CUDA cores (packed FMAs, blocks of 4 to 16) or, with TC,
// on the tcgen05 tensor cores (fd_tc.cuh; blocks of 16 to 64): M = 128 points, N = T steps,
// K = 16 rows per MMA, FP32 accumulators in tensor memory, the weights split into 16-bit hi + lo
// halves.  FP32 history on the tensor cores is stored as FP16 hi + lo planes with a power-of-two
// scale per (row, tile) (PAIR); with blocks of 32+ the near and mid units run on the tensor cores
// too, over the history's two planes (the 16-bit history stores the rounding remainder as a lo
// plane).  A tensor-core CTA runs as two independent halves (tensor memory limits a kernel to one
// CTA per SM), and a far unit may cover part of a tile (far sub-tiles) so that two halves' stages
// and accumulators fit.
// The reverse-time adjoint (ADJ) has the same structure in adjoint steps over the rows
// mu = L lambda, with a second accumulator for psi' = d psi / d gamma (see engine_kernel).
//
// Work units.  Group g holds the far units of block g (T_tiles x C x fsub: tile, chunk of R far
// rows, sub-tile; each writes T partial rows and counts itself in the tile's arrival counter)
// interleaved with the update units of block g-1 (one per step and tile, or per step and pair of
// tiles on the tensor-core kernels with many tiles; step-major): the s-th slice of block g's far
// units precedes the updates of step s, so an update is claimed only after a slice of streaming
// work, by which time its previous step is usually done.  Mid units of block g-1 precede the
// updates of steps 16, 32, 48; the group ends with block g's near units.  An update waits for
// its tile's far, near and mid counts and its halo tiles' previous step; a far unit of block g
// waits for block g-2's updates, a near or mid unit for its own tile's earlier steps.  Every wait
// therefore targets units with smaller numbers, so the persistent grid cannot deadlock whatever
// the residency.  Where the tiles are few (CUDA-core kernels), one block-long update unit per
// (block, tile) carries all of the block's steps instead (placed after one wave of block g's far
// units, which never wait for it); its sibling units must then be co-resident, which the host's
// tile limit ensures.  Determinism, bounded waits, status words and the memory-ordering protocol
// are those of engine_kernel.
#pragma once

#include <type_traits>

#include "fd_common.cuh"
#include "fd_tc.cuh"

namespace fdk {

struct UnitTB {
    int valid, inst, b, tile, chunk, C, r0, r1;
    int sub;  // far unit on the tensor cores: point range sub of the tile's fsub ranges
    int fix;  // 0: far unit; 1: update unit of step k; 2: block-long update unit; 3: near unit
    int k;
};

// Four consecutive history values of one thread's column.  The blocked kernel keeps four points
// per thread for every history type: 16 bytes of FP32, or 8 bytes of BF16 / FP16 (the FP16 rows
// carry a power-of-two scale per (row, tile), applied by the reader).
template <class TH> struct H4;
template <> struct H4<float> {
    static constexpr int BYTES = 16;
    __device__ static void unpack(float4 w, float *x)
    {
        x[0] = w.x;
        x[1] = w.y;
        x[2] = w.z;
        x[3] = w.w;
    }
    __device__ static void lds(const void *p, float *x) { unpack(*reinterpret_cast<const float4 *>(p), x); }
    __device__ static void ldg(const void *p, float *x) { unpack(__ldcg(reinterpret_cast<const float4 *>(p)), x); }
    __device__ static void stg(void *p, const float *d, float) { *reinterpret_cast<float4 *>(p) = make_float4(d[0], d[1], d[2], d[3]); }
};
template <> struct H4<__nv_bfloat16> {
    static constexpr int BYTES = 8;
    __device__ static void unpack(uint2 w, float *x)
    {
        x[0] = __uint_as_float(w.x << 16);
        x[1] = __uint_as_float(w.x & 0xffff0000u);
        x[2] = __uint_as_float(w.y << 16);
        x[3] = __uint_as_float(w.y & 0xffff0000u);
    }
    __device__ static void lds(const void *p, float *x) { unpack(*reinterpret_cast<const uint2 *>(p), x); }
    __device__ static void ldg(const void *p, float *x) { unpack(__ldcg(reinterpret_cast<const uint2 *>(p)), x); }
    __device__ static void stg(void *p, const float *d, float)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(d[0], d[1]), b = __floats2bfloat162_rn(d[2], d[3]);
        *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<unsigned *>(&a), *reinterpret_cast<unsigned *>(&b));
    }
};
template <> struct H4<__half> {
    static constexpr int BYTES = 8;
    __device__ static void unpack(uint2 w, float *x)
    {
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&w.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&w.y));
        x[0] = a.x;
        x[1] = a.y;
        x[2] = b.x;
        x[3] = b.y;
    }
    __device__ static void lds(const void *p, float *x) { unpack(*reinterpret_cast<const uint2 *>(p), x); }
    __device__ static void ldg(const void *p, float *x) { unpack(__ldcg(reinterpret_cast<const uint2 *>(p)), x); }
    // scale = 2^e per (row, tile), so the tile's largest |delta| lands in [2^14, 2^15)
    __device__ static void stg(void *p, const float *d, float scale)
    {
        __half2 a = __floats2half2_rn(d[0] * scale, d[1] * scale), b = __floats2half2_rn(d[2] * scale, d[3] * scale);
        *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<unsigned *>(&a), *reinterpret_cast<unsigned *>(&b));
    }
};

// Far rows [rlo, rhi) of block b: rows older than the previous block, within the short window.
// With adaptive memory the far rows start at the block's first settled row; the rows below
// (tail rows of some step of the block) are added by the update units.
template <int TB> __device__ __forceinline__ void far_rows(const Inst &I, int b, int &rlo, int &rhi)
{
    const int kb = b * TB;
    rhi = max(0, kb - TB);
    rlo = min(rhi, (I.mem_mode == 1) ? max(0, kb - I.mem_L) : I.gw ? I.br0[b] : 0);
}

// Adaptive memory (Definitions 3.1-3.2): lags up to e(k) carry their settled weight g(m) at step
// k (psi_m on the base interval, d psi_m at a median, 0 between medians), lags e(k)+1 .. k are
// the step's tail, weight psi_m.  e(k) from the step's schedule (nb, ng, tail_lo, tail_hi).
__device__ __forceinline__ int settled_end(const Inst &I, int k)
{
    const int4 e = I.sched[k];
    return max(e.x, e.z - 1);
}

// First row of block b's far chunks: rlo, or rlo rounded down to a multiple of I.ralign (the
// tensor-core path streams whole stages of ralign rows; rows below rlo then carry weight 0).
// rhi is a multiple of the block length, which ralign divides, so every chunk is whole stages.
template <int TB> __device__ __forceinline__ int far_origin(const Inst &I, int b)
{
    int rlo, rhi;
    far_rows<TB>(I, b, rlo, rhi);
    return I.ralign > 1 ? rlo - rlo % I.ralign : rlo;
}

// Rows per far chunk of block b: R, or enough that the block has at most cmax chunks (a multiple
// of ralign).
template <int TB> __device__ __forceinline__ int block_R(const Inst &I, int b)
{
    int rlo, rhi;
    far_rows<TB>(I, b, rlo, rhi);
    const int rows = rhi - far_origin<TB>(I, b);
    int Rb = I.cmax ? max(I.R, (rows + I.cmax - 1) / I.cmax) : I.R;
    if (I.ralign > 1) Rb = (Rb + I.ralign - 1) / I.ralign * I.ralign;
    return Rb;
}

// Far chunks of block b (at least one).
template <int TB> __device__ __forceinline__ int far_chunks(const Inst &I, int b)
{
    int rlo, rhi;
    far_rows<TB>(I, b, rlo, rhi);
    const int Rb = block_R<TB>(I, b);
    return max(1, (rhi - far_origin<TB>(I, b) + Rb - 1) / Rb);
}

// Shared state of one unit-processing CTA (the tensor-core kernels run two per CTA, see below).
struct VShared {
    Inst I;
    UnitTB U;
    int s_cur_inst, s_ok, s_ok2, s_pipe;
    int s_abort, s_iss, s_mma;
    float s_bnorm;       // FP16 tensor-core unit: power of two that scales its coefficients
    int s_ek[64];        // adaptive memory: e(k) of the block's steps
    float s_wmax[16];    // FP16 history: per-warp largest |delta| of a row
    double s_dred[16][6];  // adjoint: per-warp gradient partials
};

template <int TB, bool ADJ, class TH = float, bool TC = false>
__global__ void __launch_bounds__(512, 1) engine_tb_kernel(const Launch L)
{
    constexpr int PLANES = ADJ ? 2 : 1;
    constexpr int V = 4;  // four points per thread: a float4 of state, H4<TH> of history
    constexpr bool LOWP = sizeof(TH) == 2;
    constexpr bool F16 = std::is_same<TH, __half>::value;
    static_assert(!TC || (!ADJ && TB % 16 == 0), "tensor-core far units: forward, blocks of a multiple of 16 steps");
    // FP32 history on the tensor cores is kept as a pair of FP16 planes: row r holds
    // hi = fp16(delta 2^e) and lo = fp16(delta 2^e - hi) (about 22 significant bits together), the
    // lo plane cap rows after the hi plane; the far units multiply both (three MMAs per K slice).
    // FP16 and paired history carry a power-of-two scale 2^-e per (row, tile), which joins the
    // coefficients.
    constexpr bool PAIR = TC && !LOWP;
    constexpr bool SCALED = F16 || PAIR;
    using TB16 = typename std::conditional<SCALED, __half, __nv_bfloat16>::type;  // MMA operand type
    // A kernel holding tensor memory runs one CTA per SM, so the tensor-core kernels split each
    // CTA into two halves that work as independent CTAs: own claim loop, shared state and shared
    // memory, own named barrier, half of the CTA's tensor memory.  While one half runs an update
    // unit (latency-bound) the other keeps streaming far rows.
    constexpr int HALVES = TC ? 2 : 1;
    const int nthr = blockDim.x / HALVES;
    const int half = threadIdx.x / nthr;
    const int tid = threadIdx.x - half * nthr;
    const int RS = L.stage_rows, NS = L.stages;
    const int row_bytes = nthr * H4<TH>::BYTES;  // one history row of a tile in a stage
    // tensor cores: a stage holds RS rows of one far unit's P/fsub points (16-bit; two planes for
    // paired FP32 history)
    const int stage_tc = TC ? RS * row_bytes / L.fsub : 0;
    // units per near or mid unit's (block, tile): on the tensor cores, one per far sub-tile
    const int nsub = (TC && L.nm_tc) ? L.fsub : 1;
    // CTA (half) barriers
    auto csync = [&]() {
        if (TC)
            asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(nthr) : "memory");
        else
            __syncthreads();
    };
    auto csync_or = [&](int pred) -> int {
        if (!TC) return __syncthreads_or(pred);
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred pp, qq;\n\tsetp.ne.b32 pp, %1, 0;\n\t"
            "bar.red.or.pred qq, %2, %3, pp;\n\tselp.u32 %0, 1, 0, qq;\n\t}"
            : "=r"(r)
            : "r"(pred), "r"(1 + half), "r"(nthr)
            : "memory");
        return (int)r;
    };

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the tensor-core path's swizzled operands need 1 KB-aligned atoms; each half has its region
    unsigned char *smem = smem_raw;
    if (TC) smem += ((1024u - (tc::saddr(smem_raw) & 1023u)) & 1023u) + (size_t)half * L.smem_half;
    unsigned char *stages = smem;
    // Coefficient window in four copies shifted by 0..3 elements, so that the TB coefficients
    // of any row are TB/4 aligned 16-byte loads: copy q holds w[i + q] at index i.
    const int WS = (L.rmax + TB + 7) & ~3;                                          // copy stride
    // the stage ring also holds a block-long update unit's sums and its tile's u^k, u^{k+1}:
    // at least TB x PLANES + 2 rows of FP32 float4 columns
    // (the tensor-core kernels have no block-long update units: their ring holds the stages only)
    const size_t ring_bytes =
        TC ? (size_t)NS * stage_tc : max((size_t)NS * RS * row_bytes, (size_t)(TB * PLANES + 2) * nthr * 16);
    float *psw = reinterpret_cast<float *>(smem + ring_bytes);  // psi window
    float *psw2 = psw + 4 * WS;                                 // psi' window (ADJ)
    float *rsc = psw + PLANES * 4 * WS;                         // FP16: the far rows' scales
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(rsc + (F16 ? L.rmax : 0)) + 15) & ~uintptr_t(15));
    // Tensor-core path: after the stage ring (A operands, RS rows x P points each), a ring of NS
    // coefficient blocks (B operands, hi and lo halves side by side in TB/8 atoms), the coefficient
    // window, and the barriers: full (bulk copies landed), empty (the MMAs that read a slot are
    // done), bfull (coefficients written), done (all MMAs of a unit).
    // one coefficient block: TB/8 atoms of 8 steps x 64 K elements, hi halves at K 0..RS-1 and
    // lo halves at K RS..2RS-1 of the same rows (RS <= 32)
    constexpr int BBLK = (TB / 8) * 1024;
    unsigned char *bring = smem + ((ring_bytes + 1023) & ~(size_t)1023);
    // coefficient window and row scales cover the longest unit: a far chunk (rmax rows) or a near
    // unit (TB rows, 2 TB - 1 lags)
    const int WR = max(L.rmax, TB);
    float *win = reinterpret_cast<float *>(bring + (size_t)NS * BBLK);
    float *wsc = win + WR + TB;  // FP16 or paired history: the unit's row scales
    // tensor-core near and mid units: the settled weights of their lags (2 TB entries)
    float *win2 = wsc + (SCALED ? WR : 0);
    if (TC)
        bars = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(win2 + (L.nm_tc ? 2 * TB : 0)) + 15) & ~uintptr_t(15));
    uint64_t *full = bars, *empty = bars + NS, *bfull = bars + 2 * NS, *done_bar = bars + 3 * NS;
    __shared__ uint32_t s_tmem;
    // adaptive memory: bit j of gmask[lo] says w[lo + j] != 0 (the window of a four-row group);
    // the sparse loop reads the unshifted copy only, so the masks take the first shifted copy
    uint32_t *gmask = reinterpret_cast<uint32_t *>(psw + WS);

    static_assert(TB <= 64, "s_ek holds 64 steps");
    __shared__ VShared vsh[HALVES];
    VShared &VS = vsh[half];
    Inst &I = VS.I;
    UnitTB &U = VS.U;
    int &s_cur_inst = VS.s_cur_inst, &s_ok = VS.s_ok, &s_ok2 = VS.s_ok2, &s_pipe = VS.s_pipe;
    int &s_abort = VS.s_abort, &s_iss = VS.s_iss, &s_mma = VS.s_mma;
    float &s_bnorm = VS.s_bnorm;
    int *s_ek = VS.s_ek;
    float *s_wmax = VS.s_wmax;
    double(*s_dred)[6] = VS.s_dred;

    if (tid == 0) {
        if (TC) {
            for (int b = 0; b < NS; ++b) {
                mbar_init(&full[b], 1);
                mbar_init(&empty[b], 1);
                mbar_init(&bfull[b], (uint32_t)(nthr - 64));
            }
            mbar_init(done_bar, 1);
        } else {
            for (int b = 0; b < NS; ++b) mbar_init(&bars[b], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_cur_inst = -1;
    }
    // tensor memory for the far accumulators: P/128 blocks of TB FP32 columns per half (tc_cols,
    // a power of two), allocated once per CTA (one CTA per SM)
    const uint32_t tc_cols = TC ? (uint32_t)L.inst[0].tc_cols : 0u;
    if (TC && (tc_cols < 32u || (tc_cols & (tc_cols - 1u)) || tc_cols * HALVES > 512u)) {
        // not an allocatable column count: report and leave before any barrier (uniform)
        if (threadIdx.x == 0) atomicCAS(L.err, ERR_NONE, ERR_PIPE);
        return;
    }
    if (TC && threadIdx.x < 32) tc::tmem_alloc(&s_tmem, tc_cols * HALVES);
    if (TC) tc::fence_before();
    __syncthreads();
    if (TC) tc::fence_after();
    const uint32_t tmem = TC ? s_tmem + (uint32_t)half * tc_cols : 0u;
    uint32_t tc_use = 0, tc_done = 0;  // stages streamed and units finished by this CTA (TC)

    uint32_t n_issued = 0, n_used = 0;
    int ghint = L.g_begin;
    // thread 0: the group of the last claimed unit (units [cg_lo, cg_hi), info cgi), so that a
    // claim in the same group reads no group table
    long long cg_lo = 0, cg_hi = 0;
    int2 cgi = make_int2(0, 0);
    const long long u_base = L.g_off[L.g_begin];
    const long long u_end = L.g_off[L.g_end];

    for (;;) {
        // ---------------------------------------------------------------- claim
        // Thread 0 passes over units with nothing to do in this launch (far units of a block
        // that starts at or after the launch's end, updates of steps outside it) without
        // publishing them: every published unit ends with a CTA barrier, so the shared
        // descriptor is never rewritten while another thread may still read it.
        if (tid == 0) {
            int ok = 0;
            for (;;) {
                // claimed when needed, never ahead: a CTA waiting inside a block-long update unit
                // must not hold an unstarted unit that its neighbours' units wait for
                // (the status word is read before the queue add, so the two latencies overlap)
                const int err_now = ld_volatile(L.err);
                const long long u = u_base + (long long)atomicAdd(L.queue, 1ull);
                ok = (u < u_end) && (err_now == ERR_NONE);
                if (!ok) break;
                if (u < cg_lo || u >= cg_hi) {
                    const int g = find_group(L.g_off, ghint, L.g_end, u);
                    ghint = g;
                    cg_lo = L.g_off[g];
                    cg_hi = L.g_off[g + 1];
                    cgi = L.g_info[g];
                }
                const int2 gi = cgi;
                if (gi.x != s_cur_inst) {
                    I = L.inst[gi.x];
                    s_cur_inst = gi.x;
                }
                const long long local = u - cg_lo, gsize = cg_hi - cg_lo;
                const int gb = gi.y;  // group: far units of block gb, updates of block gb-1
                const int k_end = min(L.k_end, I.ksteps);  // a batch runs each instance to its end
                // block gb-1's update units: per (block, tile), or per (step, group of ug tiles)
                const int Tu = (gb >= 1) ? (I.ub ? I.T : (I.T + I.ug - 1) / I.ug * TB) : 0;
                const int Mu = (gb >= 1) ? I.T * I.mid * nsub : 0;       // block gb-1's mid units
                const long long F = gsize - (long long)(Tu + Mu);  // block gb's far units
                long long f = -1;  // far unit index within block gb, or -1 for an update unit
                U.inst = gi.x;
                if (I.ub) {
                    // About one wave of block gb's far units (as many as the CTAs that the update
                    // units leave), then block gb-1's block-long update units, then the rest of
                    // block gb's far units.  An update unit is claimed when block gb-1's far
                    // units are about to finish instead of holding its SM through their tail;
                    // block gb's far units read rows up to block gb-2 only, so none of them
                    // waits for these updates.
                    const long long F1 = min(F, (long long)max(0, (int)gridDim.x * HALVES - Tu));
                    if (local >= F1 && local < F1 + Tu) {
                        const int kb1 = (gb - 1) * TB;
                        if (max(kb1, L.k0) >= min(kb1 + TB, k_end)) continue;  // no step in this launch
                        U.fix = 2;
                        U.b = gb - 1;
                        U.tile = (int)(local - F1);
                        U.k = 0;
                        U.C = far_chunks<TB>(I, gb - 1);
                        U.chunk = 0;
                        U.r0 = U.r1 = 0;
                    } else {
                        f = (local < F1) ? local : local - Tu;
                    }
                } else if (I.near && gb * TB < I.ksteps && local >= gsize - I.T * nsub) {
                    // near unit of block gb (the group's last T units): the previous block's rows
                    // for every step of block gb, once block gb-1's updates of the tile are done
                    const int kb = gb * TB;
                    if (kb >= k_end) continue;  // block starts at or after the launch's end
                    U.fix = 3;
                    U.b = gb;
                    const int nidx = (int)(local - (gsize - I.T * nsub));
                    U.tile = nidx % I.T;
                    U.sub = nidx / I.T;
                    U.C = far_chunks<TB>(I, gb);
                    U.chunk = U.C;  // its partial rows follow the far chunks'
                    U.r0 = max(0, kb - TB);
                    U.r1 = kb;
                    U.k = 0;
                    if (kb - L.k0 > 0) {
                        const int w = wait_until(&I.done[U.tile], (unsigned)(kb - L.k0), L, 512);
                        if (w < 0) note_failure(L, 12, gb, U.tile, kb - L.k0, ld_acquire(&I.done[U.tile]), L.k0, 0);
                        if (w <= 0) ok = 0;
                    }
                    break;
                } else {
                    // segment s: far slice s, then (s = 16 j, j = 1 .. mid) the T mid units of
                    // sub-block j of block gb-1, then the T update units of step s
                    int sseg = 0;
                    const int Ts = Tu / TB;
                    const long long F0 = F - (I.near && gb * TB < I.ksteps ? I.T * nsub : 0);  // far units proper
                    auto seg_start = [&](int sg) -> long long {
                        const int mids = (Mu && sg >= 1) ? min(I.mid, (sg - 1) / 16) : 0;
                        return (long long)sg * Ts + (long long)I.T * nsub * mids + (long long)sg * F0 / TB;
                    };
                    // segments are near equal: estimate, then step to the exact one
                    sseg = (int)min((long long)(TB - 1), local * TB / max(1ll, (long long)TB * Ts + F0 + Mu));
                    while (sseg > 0 && seg_start(sseg) > local) --sseg;
                    while (sseg + 1 < TB && seg_start(sseg + 1) <= local) ++sseg;
                    const long long fs0 = (long long)sseg * F0 / TB;
                    const long long fsn = (long long)(sseg + 1) * F0 / TB - fs0;  // far units in slice s
                    long long off = local - seg_start(sseg);
                    const bool seg_mid = Mu && sseg >= 16 && sseg % 16 == 0;
                    if (seg_mid && off >= fsn && off < fsn + I.T * nsub) {
                        // mid unit: rows kb .. kb+s-1 of block gb-1 for its steps s .. s+15.  Skipped
                        // only when no update of this launch needs it (the updates' arrival target
                        // counts every earlier sub-block's mid unit, so those run even when their
                        // own steps precede the launch).
                        const int kb1 = (gb - 1) * TB;
                        if (kb1 + sseg >= k_end || kb1 + TB <= L.k0) continue;
                        U.fix = 4;
                        U.b = gb - 1;
                        U.tile = (int)((off - fsn) % I.T);
                        U.sub = (int)((off - fsn) / I.T);
                        U.k = kb1 + sseg;
                        U.C = far_chunks<TB>(I, gb - 1);
                        U.chunk = U.C + 1;  // after the far chunks' and the near unit's rows
                        U.r0 = kb1;
                        U.r1 = kb1 + sseg;
                        if (U.r1 - L.k0 > 0) {  // the tile's rows up to r1-1 written
                            const int w = wait_until(&I.done[U.tile], (unsigned)(U.r1 - L.k0), L, 512);
                            if (w < 0) note_failure(L, 13, gb, U.tile, U.r1 - L.k0, ld_acquire(&I.done[U.tile]), L.k0, 0);
                            if (w <= 0) ok = 0;
                        }
                        break;
                    }
                    if (seg_mid && off >= fsn) off -= I.T * nsub;
                    if (off >= fsn) {  // update unit: block gb-1, step s
                        const int k = (gb - 1) * TB + sseg;
                        if (k < L.k0 || k >= k_end) continue;  // block edge outside this launch
                        U.fix = 1;
                        U.b = gb - 1;
                        U.tile = (int)(off - fsn) * I.ug;
                        U.k = k;
                        U.C = far_chunks<TB>(I, gb - 1);
                        U.chunk = 0;
                        U.r0 = U.r1 = 0;
                    } else {
                        f = fs0 + off;
                    }
                }
                if (f >= 0) {  // far unit of block gb
                    const int kb = gb * TB;
                    if (kb >= k_end) continue;  // block starts at or after the launch's end
                    int rlo, rhi;
                    far_rows<TB>(I, gb, rlo, rhi);
                    const int Rb = block_R<TB>(I, gb);
                    U.fix = 0;
                    U.b = gb;
                    U.C = far_chunks<TB>(I, gb);
                    U.tile = (int)(f % I.T);
                    U.sub = (int)((f / I.T) % L.fsub);
                    U.chunk = (int)(f / I.T / L.fsub);
                    U.r0 = min(rhi, far_origin<TB>(I, gb) + U.chunk * Rb);
                    U.r1 = min(rhi, U.r0 + Rb);
                    U.k = 0;
                    // far rows up to r1-1 written (block-long units: their whole block, whose
                    // last step fences the block's rows for bulk copies); partial rows of block
                    // b-npar consumed
                    int need = 0;
                    if (U.r1 > U.r0) need = (I.ub ? (U.r1 + TB - 1) / TB * TB : U.r1) - L.k0;
                    need = max(need, kb - (I.npar - 1) * TB - L.k0);
                    if (need > 0) {
                        const int w = wait_until(&I.done[U.tile], (unsigned)need, L, 512);
                        if (w < 0) note_failure(L, 1, gb, U.tile, need, ld_acquire(&I.done[U.tile]), L.k0, 0);
                        if (w <= 0) ok = 0;
                    }
                }
                break;
            }
            U.valid = ok;
        }
        csync();
        if (!U.valid) break;

        int tile = U.tile;  // (a per-step update unit of several tiles moves it from tile to tile)
        const int C = U.C, b = U.b, kb = b * TB;
        const int par = b % I.npar;
        // Arrival counters carry the block's generation within its parity in the high half
        // ((b - the launch's first block k0/TB) / npar), so a count left by block b - npar can never
        // satisfy block b's wait; the last update of block b sets the word for block b + npar.
        auto arrive_target = [&](int bb, int count) -> unsigned {
            return ((unsigned)((bb - L.k0 / TB) / I.npar) << 16) + (unsigned)count;
        };
        int j0 = tile * I.P + tid * V;
        auto prow = [&](int c, int t, int plane) -> float * {
            return reinterpret_cast<float *>(I.part +
                                             ((size_t)(((par * I.maxC + c) * TB + t) * PLANES + plane)) * I.part_pitch);
        };

        if (!U.fix || (TC && L.nm_tc && (U.fix == 3 || U.fix == 4))) {
            if constexpr (TC) {
                // ============================================== far unit on the tensor cores
                // (and, with blocks of 32 or more, the near and mid units: the same contraction over
                // the previous block's rows for the block's steps, or over the block's earlier rows
                // for one sub-block's 16 steps, from the history's hi and lo planes: the pair of
                // paired FP32 history, or the 16-bit row and its rounding remainder)
                // D[p][t] = sum over rows r in [r0, r1) of H[r][p] * c(t, r), c(t, r) = w(kb + t - r):
                // M = 128 points, N = TB steps, K = 16 rows per MMA, FP32 accumulators in tensor
                // memory (block m of the unit's Pf/128 point blocks at columns m*TB ...; the unit
                // covers the tile's points sub*Pf .. (sub+1)*Pf-1, Pf = P/fsub).  The
                // weights are split into 16-bit hi + lo halves (two MMAs per K slice), so they keep
                // about 16 (BF16) or 22 (FP16) significant bits; paired FP32 history adds its lo
                // plane (a third MMA).  Roles: warp 0 lane 0 issues the tensor-map copies of the
                // history stages, warp 1 lane 0 issues the MMAs, the other warps write each
                // stage's coefficient block; mbarriers order them, with no CTA barrier per stage.
                const bool nm = U.fix != 0;                    // near or mid unit
                // near and mid units read both planes in stages of 16 rows (as paired far units
                // do), 16-bit far units one plane in stages of RS rows: the same bytes per stage
                const bool two = PAIR || nm;
                const int RSu = nm ? 16 : RS;
                const void *tmu = (nm && !PAIR) ? I.tmap2 : I.tmap;
                const int rank_u = (nm && !PAIR) ? I.tmap2_rank : I.tmap_rank;
                const int r0 = U.r0, r1 = U.r1, nrow = r1 - r0;  // whole stages (multiples of RSu)
                const int nst = nrow / RSu;
                const int warp = tid >> 5, lane = tid & 31, nwarp = nthr >> 5;
                const int Pf = I.P / L.fsub, p0 = tile * I.P + U.sub * Pf;  // the unit's points
                const int MB = Pf / 128;
                const int t_lo = (U.fix == 4) ? U.k - kb : 0;  // its steps: kb+t_lo .. kb+t_lo+NN-1
                const int NN = (U.fix == 4) ? 16 : TB;
                // near and mid rows take each step's own weight of their lag (adaptive memory: the
                // settled weight up to the step's e(k), psi beyond), far rows the settled one
                const bool per_step = nm && I.gw;
                int rlo_t, rhi_t;
                far_rows<TB>(I, b, rlo_t, rhi_t);  // rows below rlo_t are not far rows of this block
                if (nm) rlo_t = r0;
                {
                    // coefficient window win[j] = w(lag0 + j), lag0 = kb + t_lo - (r1 - 1): row r,
                    // step kb+t_lo+t uses win[(r1 - 1 - r) + t]; short memory cuts lags beyond its
                    // window; per-step weights take win (psi) or win2 (settled) by the step's e(k)
                    const float *wsrc = reinterpret_cast<const float *>((I.gw && !nm) ? I.gw : I.psi);
                    const int lag0 = kb + t_lo - (r1 - 1);
                    float amax = 0.f, smax = 0.f;
                    for (int j = tid; j < nrow + NN - 1; j += nthr) {
                        const int lag = lag0 + j;
                        const bool cut = I.mem_mode == 1 && lag > I.mem_L;
                        win[j] = cut ? 0.f : wsrc[lag];
                        amax = fmaxf(amax, fabsf(win[j]));
                        if (per_step) {
                            win2[j] = cut ? 0.f : reinterpret_cast<const float *>(I.gw)[lag];
                            amax = fmaxf(amax, fabsf(win2[j]));
                        }
                    }
                    if (per_step && tid < TB) s_ek[tid] = (kb + tid < I.ksteps) ? settled_end(I, kb + tid) : 0x7fffffff;
                    if (SCALED) {
                        // FP16 rows hold delta * 2^e per (row, tile) (paired rows their hi and lo
                        // parts): the row's scale 2^-e joins its weights, and one power of two per
                        // unit keeps every coefficient below 2^14, so the FP16 halves cannot
                        // overflow; the epilogue divides it out.  The bound is (largest weight) x
                        // (largest row scale) over the whole unit: the two maxima are reduced
                        // separately, as the largest weight and the largest scale may sit in
                        // different threads' shares.
                        for (int a = tid; a < nrow; a += nthr) {
                            wsc[a] = __ldcg(I.hscale + (size_t)((r0 + a) % I.cap) * I.T + tile);
                            smax = fmaxf(smax, wsc[a]);
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                            smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
                        }
                        if ((tid & 31) == 0) {  // (at most 8 warps per half: 256 threads)
                            s_wmax[tid >> 5] = amax;
                            s_wmax[8 + (tid >> 5)] = smax;
                        }
                    }
                    if (tid == 0) {
                        s_abort = 0;
                        s_iss = 0;
                        s_mma = 0;
                    }
                }
                csync();
                if (SCALED) {
                    if (tid == 0) {
                        float am = 0.f, sm = 0.f;
                        for (int w = 0; w < nthr / 32; ++w) {
                            am = fmaxf(am, s_wmax[w]);
                            sm = fmaxf(sm, s_wmax[8 + w]);
                        }
                        const float m = am * sm;
                        int ex = 0;
                        if (m > 0.f && isfinite(m)) frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
                        s_bnorm = ldexpf(1.f, max(-120, min(120, 14 - ex)));
                    }
                    csync();
                }
                const float bnorm = SCALED ? s_bnorm : 1.f, binv = 1.f / bnorm;  // powers of two
                auto give_up = [&](int site_s, uint64_t *bar) {
                    if (atomicCAS(L.err, ERR_NONE, ERR_PIPE) == ERR_NONE)
                        note_failure(L, 11, ((long long)b << 32) | tile, ((long long)site_s << 32) | nst,
                                     (long long)tc_use, (long long)*reinterpret_cast<volatile unsigned long long *>(bar),
                                     ((long long)L.k0 << 32) | L.k_end, ((long long)r0 << 32) | r1);
                    atomicExch(&s_abort, 1);
                };
                // bounded wait for an mbarrier phase; false when it gave up (or another role did)
                auto wait_bar = [&](uint64_t *bar, uint32_t parity, int site_s) -> bool {
                    if (mbar_try_wait(bar, parity)) return true;
                    const long long t0 = globaltimer();
                    while (!mbar_try_wait(bar, parity)) {
                        if (*reinterpret_cast<volatile int *>(&s_abort)) return false;
                        if (globaltimer() - t0 > L.timeout_ns) {
                            give_up(site_s, bar);
                            return false;
                        }
                    }
                    return true;
                };
                constexpr uint32_t IDESC = tc::idesc_f16_amn(128, TB, !SCALED);
                constexpr uint32_t IDESC16 = tc::idesc_f16_amn(128, 16, !SCALED);  // mid units
                const uint32_t idesc = (NN == TB) ? IDESC : IDESC16;
                if (warp == 0) {
                    if (lane == 0) {  // history stages: 64 points x RS rows per point group
                        // (two planes: the hi plane's box, then the lo plane's, cap rows on)
                        const size_t plane_bytes = (size_t)RSu * Pf * 2;
                        for (int s = 0; s < nst; ++s) {
                            const uint32_t use = tc_use + (uint32_t)s, slot = use % (uint32_t)NS;
                            if (!wait_bar(&empty[slot], ((use / (uint32_t)NS) & 1u) ^ 1u, s)) break;
                            unsigned char *a = stages + (size_t)slot * stage_tc;
                            mbar_expect_tx(&full[slot], (uint32_t)stage_tc);
                            for (int pl = 0; pl < (two ? 2 : 1); ++pl) {
                                unsigned char *ap = a + pl * plane_bytes;
                                const int y = r0 + s * RSu + pl * I.cap;
                                if (rank_u == 3)  // one box: 64 points x RSu rows x Pf/64 point groups
                                    tc::tma_load_3d(ap, tmu, 0, y, p0 / 64, &full[slot]);
                                else
                                    for (int j = 0; j < Pf / 64; ++j)
                                        tc::tma_load_2d(ap + (size_t)j * RSu * 128, tmu, p0 + 64 * j, y,
                                                        &full[slot]);
                            }
                            s_iss = s + 1;
                        }
                    }
                } else if (warp == 1) {
                    if (lane == 0) {
                        for (int s = 0; s < nst; ++s) {
                            const uint32_t use = tc_use + (uint32_t)s, slot = use % (uint32_t)NS;
                            const uint32_t ph = (use / (uint32_t)NS) & 1u;
                            if (!wait_bar(&full[slot], ph, s) || !wait_bar(&bfull[slot], ph, s)) break;
                            tc::fence_after();
                            const uint32_t a0 = tc::saddr(stages + (size_t)slot * stage_tc);
                            const uint32_t bh = tc::saddr(bring + (size_t)slot * BBLK), bl = bh + (uint32_t)(RSu * 2);
                            if (two) {
                                // A: hi plane as below, the lo plane RSu*Pf*2 bytes further
                                const uint32_t lo_off = (uint32_t)(RSu * Pf * 2);
                                for (int m = 0; m < MB; ++m)
                                    for (int kk = 0; kk < RSu / 16; ++kk) {
                                        const uint32_t ah = a0 + (uint32_t)(2 * m * RSu * 128 + kk * 2048);
                                        const uint64_t dh = tc::desc_sw128(ah, (uint32_t)(RSu * 128), 1024u);
                                        const uint64_t dl = tc::desc_sw128(ah + lo_off, (uint32_t)(RSu * 128), 1024u);
                                        const uint32_t d = tmem + (uint32_t)(m * TB);
                                        const uint32_t acc = (s | kk) ? 1u : 0u;
                                        const uint64_t bdh = tc::desc_sw128(bh + (uint32_t)(kk * 32), 16u, 1024u);
                                        tc::mma_f16(d, dh, bdh, idesc, acc);
                                        tc::mma_f16(d, dh, tc::desc_sw128(bl + (uint32_t)(kk * 32), 16u, 1024u), idesc, 1u);
                                        tc::mma_f16(d, dl, bdh, idesc, 1u);
                                    }
                            } else
                            for (int m = 0; m < MB; ++m)
                                for (int kk = 0; kk < RS / 16; ++kk) {
                                    // A: points 128m.., rows 16kk..; atoms of 64 points are RS*128
                                    // bytes apart (LBO), atoms of 8 rows 1 KB apart (SBO)
                                    const uint64_t ad = tc::desc_sw128(a0 + (uint32_t)(2 * m * RS * 128 + kk * 2048),
                                                                       (uint32_t)(RS * 128), 1024u);
                                    const uint32_t d = tmem + (uint32_t)(m * TB);
                                    const uint32_t acc = (s | kk) ? 1u : 0u;
                                    tc::mma_f16(d, ad, tc::desc_sw128(bh + (uint32_t)(kk * 32), 16u, 1024u), idesc, acc);
                                    tc::mma_f16(d, ad, tc::desc_sw128(bl + (uint32_t)(kk * 32), 16u, 1024u), idesc, 1u);
                                }
                            tc::commit(&empty[slot]);  // the slot is free once these MMAs are done
                            s_mma = s + 1;
                        }
                        if (nst > 0) tc::commit(done_bar);  // every MMA this unit issued
                    }
                } else {
                    // coefficient blocks, K-major with the 128-byte swizzle: step t is row t of the
                    // block (atom t/8, row t%8), stage row i its K index
                    const int nb = nthr - 64, me = tid - 64;
                    for (int s = 0; s < nst; ++s) {
                        const uint32_t use = tc_use + (uint32_t)s, slot = use % (uint32_t)NS;
                        if (!wait_bar(&empty[slot], ((use / (uint32_t)NS) & 1u) ^ 1u, s)) break;
                        unsigned char *bh = bring + (size_t)slot * BBLK;
                        for (int e = me; e < NN * RSu; e += nb) {
                            const int t = e / RSu, i = e - t * RSu;
                            const int r = r0 + s * RSu + i;
                            const int wi = (r1 - 1 - r) + t;
                            float c = (r < rlo_t) ? 0.f
                                      : (per_step && kb + t_lo + t - r <= s_ek[t_lo + t]) ? win2[wi]
                                                                                         : win[wi];
                            if (SCALED) c *= wsc[r - r0] * bnorm;
                            TB16 hi, lo;
                            if constexpr (SCALED) {
                                hi = __float2half_rn(c);
                                lo = __float2half_rn(c - __half2float(hi));
                            } else {
                                hi = __float2bfloat16_rn(c);
                                lo = __float2bfloat16_rn(c - __bfloat162float(hi));
                            }
                            const int row = t & 7, base = (t >> 3) * 1024 + row * 128;
                            auto off = [&](int kq) { return base + (((kq >> 3) ^ row) << 4) + (kq & 7) * 2; };
                            *reinterpret_cast<TB16 *>(bh + off(i)) = hi;
                            *reinterpret_cast<TB16 *>(bh + off(RSu + i)) = lo;
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(&bfull[slot])) : "memory");
                    }
                }
                __syncwarp();  // warps 0 and 1: the other lanes wait for lane 0's loop
                csync();
                if (s_abort) {
                    // stop: wait (bounded) for the copies and MMAs already issued, then leave
                    if (tid == 32 && s_mma > 0) {
                        const long long t0 = globaltimer();
                        while (!mbar_try_wait(done_bar, tc_done & 1u) && globaltimer() - t0 < L.timeout_ns) {
                        }
                    }
                    if (tid == 0) {
                        const long long t0 = globaltimer();
                        for (int s = s_mma; s < s_iss; ++s) {
                            const uint32_t use = tc_use + (uint32_t)s, slot = use % (uint32_t)NS;
                            while (!mbar_try_wait(&full[slot], (use / (uint32_t)NS) & 1u) &&
                                   globaltimer() - t0 < L.timeout_ns) {
                            }
                        }
                    }
                    csync();
                    break;
                }
                tc_use += (uint32_t)nst;
                if (nst > 0) {
                    if (!mbar_try_wait(done_bar, tc_done & 1u)) {
                        const long long t0 = globaltimer();
                        while (!mbar_try_wait(done_bar, tc_done & 1u))
                            if (globaltimer() - t0 > L.timeout_ns) {
                                give_up(nst, done_bar);
                                break;
                            }
                    }
                    ++tc_done;
                }
                tc::fence_after();
                // chunk c stores the running sum S_c = S_{c-1} + p_c with block-long update units
                const int c0 = U.chunk;
                const bool chain = I.ub && c0 > 0;
                if (chain && tid == 0) {
                    const int w = wait_until(&I.arrive[par * I.T + tile], arrive_target(b, c0), L, 512);
                    if (w < 0) note_failure(L, 10, b, tile, arrive_target(b, c0), ld_acquire(&I.arrive[par * I.T + tile]), L.k0, 0);
                    if (w <= 0) atomicExch(&s_abort, 1);
                }
                csync();
                if (s_abort) break;
                // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. of point blocks
                // m = w / 4, w / 4 + nwarp / 4, ...; each thread takes one point's NN sums, 16
                // columns at a time
                const int q = warp & 3;
                for (int m = warp >> 2; m < MB; m += nwarp >> 2) {
                    const int j = p0 + m * 128 + q * 32 + lane;
#pragma unroll 1
                    for (int c = 0; c < NN; c += 16) {  // warp-uniform
                        float v[16];
                        if (nst > 0) {
                            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(m * TB + c), v);
                        } else {
#pragma unroll
                            for (int t = 0; t < 16; ++t) v[t] = 0.f;
                        }
                        if (SCALED) {  // exact: a power of two
#pragma unroll
                            for (int t = 0; t < 16; ++t) v[t] *= binv;
                        }
                        if (j < I.N) {
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                float sum = v[t];
                                if (chain) sum = __ldcg(prow(c0 - 1, c + t, 0) + j) + v[t];
                                prow(c0, t_lo + c + t, 0)[j] = sum;
                            }
                        }
                    }
                }
                // CTA barrier, then one release add: cumulative over every thread's partial stores
                tc::fence_before();
                csync();
                if (tid == 0) atom_add_acq_rel(&I.arrive[par * I.T + tile], 1u);
                continue;
            } else {
                // ================================================================ far unit
                const int r0 = U.r0, r1 = U.r1, nrow = r1 - r0;
                const int nst = (nrow + RS - 1) / RS;
                long long tile_bytes = (long long)min(I.P, I.N - tile * I.P) * (long long)sizeof(TH);
                tile_bytes = (tile_bytes + 15) & ~15ll;

                // coefficient window w[i] = psi_{lag0 + i}: row r, step kb+t uses w[(r1-1-r) + t]
                const bool sparse = !ADJ && I.gw != nullptr;
                {
                    const float *psi = reinterpret_cast<const float *>(I.psi);
                    const int lag0 = kb - (r1 - 1);
                    const int nw = nrow + TB - 1;
                    for (int e = tid; e < (sparse ? WS : 4 * WS); e += nthr) {
                        const int q = e / WS, i = e - q * WS, w = i + q;
                        const int lag = lag0 + w;
                        const bool cut = (w >= nw) || (I.mem_mode == 1 && lag > I.mem_L);
                        psw[q * WS + i] = cut ? 0.f : I.gw ? reinterpret_cast<const float *>(I.gw)[lag] : psi[lag];
                        if (ADJ) psw2[q * WS + i] = cut ? 0.f : reinterpret_cast<const float *>(I.dpsi)[lag];
                    }
                }
                csync();
                // Adaptive memory: the settled weights are zero between medians (at least two of three
                // lags in the far rows), so a four-row group multiplies only the lags its window holds.
                if (sparse) {
                    for (int lo = tid; lo + 4 <= nrow; lo += nthr) {
                        uint32_t m = 0;
                        for (int j = 0; j < TB + 4; ++j) m |= (psw[lo + j] != 0.f ? 1u : 0u) << j;
                        gmask[lo] = m;
                    }
                    csync();
                }

                // FP16 history: the power-of-two scale of each far row on this tile
                if (F16) {
                    for (int a = tid; a < nrow; a += nthr)
                        rsc[a] = __ldcg(I.hscale + (size_t)((r0 + a) % I.cap) * I.T + tile);
                    csync();
                }

                // accumulators as point pairs: one packed two-lane FMA (each lane an IEEE fmaf)
                // serves two points, halving the far loop's FMA instructions
                float2 acc[TB][V / 2], acc2[ADJ ? TB : 1][V / 2];
    #pragma unroll
                for (int t = 0; t < TB; ++t)
    #pragma unroll
                    for (int h = 0; h < V / 2; ++h) acc[t][h] = make_float2(0.f, 0.f);
    #pragma unroll
                for (int t = 0; t < (ADJ ? TB : 1); ++t)
    #pragma unroll
                    for (int h = 0; h < V / 2; ++h) acc2[t][h] = make_float2(0.f, 0.f);

                // Stage s is filled by warp s mod (warps), one lane per row: the copies of a stage
                // go out together and the issue work rotates over the warps instead of delaying
                // one warp at every stage barrier.  Called by all lanes of the issuing warp.
                const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
                auto issue = [&](int s, uint32_t slot) {
                    const int bb = (int)(slot % (uint32_t)NS);
                    const int a0 = s * RS, a1 = min(nrow, a0 + RS);
                    if (lane == 0) mbar_expect_tx(&bars[bb], (uint32_t)(tile_bytes * (a1 - a0)));
                    __syncwarp();
                    const char *col = I.hist + (size_t)tile * I.P * sizeof(TH);
                    for (int a = a0 + lane; a < a1; a += 32)
                        bulk_g2s(stages + ((size_t)bb * RS + (a - a0)) * row_bytes,
                                 col + (size_t)((r0 + a) % I.cap) * I.pitch, (uint32_t)tile_bytes, &bars[bb]);
                };
                // every lane that issues copies orders the rows it acquired before the async proxy
                if (lane < RS) fence_proxy_async_global();
                {
                    const int pre = min(NS, nst);
                    for (int s = 0; s < pre; ++s)
                        if (warp == s % nwarp) issue(s, n_issued + (uint32_t)s);
                    n_issued += (uint32_t)pre;
                }
                int aborted = 0;
                for (int s = 0; s < nst; ++s) {
                    const int bb = (int)(n_used % (uint32_t)NS);
                    const uint32_t ph = (n_used / (uint32_t)NS) & 1u;
                    int tmo = 0;
                    if (!mbar_try_wait(&bars[bb], ph)) {
                        const long long t0 = globaltimer();
                        while (!mbar_try_wait(&bars[bb], ph)) {
                            if (globaltimer() - t0 > L.timeout_ns) {
                                if (atomicCAS(L.err, ERR_NONE, ERR_PIPE) == ERR_NONE)
                                    note_failure(L, 2, ((long long)b << 32) | tile, ((long long)s << 32) | nst,
                                                 ((long long)n_issued << 32) | n_used,
                                                 (long long)*reinterpret_cast<volatile unsigned long long *>(&bars[bb]),
                                                 ((long long)L.k0 << 32) | L.k_end, ((long long)r0 << 32) | r1);
                                tmo = 1;  // the copy is still owed to this slot; see below
                                break;
                            }
                        }
                    }
                    const int rows = tmo ? 0 : min(RS, nrow - s * RS);
                    const unsigned char *base = stages + (size_t)bb * RS * row_bytes + (size_t)tid * H4<TH>::BYTES;
                    // row a of the unit (a = s*RS + row within the stage), converted to FP32
                    auto ldrow = [&](int rr, float *x) {
                        H4<TH>::lds(base + (size_t)rr * row_bytes, x);
                        if (F16) {
                            const float sc = rsc[s * RS + rr];
    #pragma unroll
                            for (int v = 0; v < V; ++v) x[v] *= sc;
                        }
                    };
                    int r = 0;
                    if (sparse) {
                        // Four rows at a time, lag by lag over the window's nonzero weights only.  Lag
                        // J of the window meets row i at step t = J - 3 + i; J descending keeps each
                        // accumulator's rows in increasing order, as in the dense loop below, and the
                        // skipped products are exact zeros, so the sums are the dense loop's.
                        for (; r + 4 <= rows; r += 4) {
                            const int lo = nrow - 1 - (s * RS + r) - 3;
                            const uint32_t m = gmask[lo];
                            float x[4][V];
    #pragma unroll
                            for (int i = 0; i < 4; ++i) ldrow(r + i, x[i]);
    #pragma unroll
                            for (int J = TB + 3; J >= 0; --J) {
                                if (!(m & (1u << J))) continue;
                                const float cj = psw[lo + J];
                                const float2 cj2 = make_float2(cj, cj);
    #pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const int t = J - 3 + i;
                                    if (t < 0 || t >= TB) continue;
    #pragma unroll
                                    for (int h = 0; h < V / 2; ++h)
                                        acc[t][h] = __ffma2_rn(cj2, make_float2(x[i][2 * h], x[i][2 * h + 1]), acc[t][h]);
                                }
                            }
                        }
                    }
                    // Four rows at a time.  Row a = s*RS + r + i uses w[wo - i + t], wo = nrow-1-(s*RS+r):
                    // the TB+3 coefficients w[wo-3 .. wo+TB-1] come in aligned 16-byte loads from the
                    // copy shifted by (wo-3) & 3 and serve all four rows from registers.
                    for (; r + 4 <= rows; r += 4) {
                        const int lo = nrow - 1 - (s * RS + r) - 3;
                        const int cq = (lo & 3) * WS + (lo & ~3);
                        float c[TB + 4], c2[ADJ ? TB + 4 : 1];
    #pragma unroll
                        for (int j = 0; j < TB + 4; j += 4) {
                            const float4 c4 = *reinterpret_cast<const float4 *>(psw + cq + j);
                            c[j] = c4.x;
                            c[j + 1] = c4.y;
                            c[j + 2] = c4.z;
                            c[j + 3] = c4.w;
                            if (ADJ) {
                                const float4 d4 = *reinterpret_cast<const float4 *>(psw2 + cq + j);
                                c2[ADJ ? j : 0] = d4.x;
                                c2[ADJ ? j + 1 : 0] = d4.y;
                                c2[ADJ ? j + 2 : 0] = d4.z;
                                c2[ADJ ? j + 3 : 0] = d4.w;
                            }
                        }
    #pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float x[4];
                            ldrow(r + i, x);
    #pragma unroll
                            for (int t = 0; t < TB; ++t)
    #pragma unroll
                                for (int h = 0; h < V / 2; ++h)
                                    acc[t][h] = __ffma2_rn(make_float2(c[3 - i + t], c[3 - i + t]), make_float2(x[2 * h], x[2 * h + 1]),
                                                           acc[t][h]);
                            if (ADJ) {
    #pragma unroll
                                for (int t = 0; t < (ADJ ? TB : 1); ++t)
    #pragma unroll
                                    for (int h = 0; h < V / 2; ++h)
                                        acc2[t][h] = __ffma2_rn(make_float2(c2[ADJ ? 3 - i + t : 0], c2[ADJ ? 3 - i + t : 0]),
                                                                make_float2(x[2 * h], x[2 * h + 1]), acc2[t][h]);
                            }
                        }
                    }
                    for (; r < rows; ++r) {  // remaining rows one at a time (unshifted copy)
                        float x[4];
                        ldrow(r, x);
                        const int wo = nrow - 1 - (s * RS + r);
    #pragma unroll
                        for (int t = 0; t < TB; ++t) {
                            const float cc = psw[wo + t];
    #pragma unroll
                            for (int h = 0; h < V / 2; ++h)
                                acc[t][h] = __ffma2_rn(make_float2(cc, cc), make_float2(x[2 * h], x[2 * h + 1]), acc[t][h]);
                            if (ADJ) {
                                const float cd = psw2[wo + t];
    #pragma unroll
                                for (int h = 0; h < V / 2; ++h)
                                    acc2[ADJ ? t : 0][h] = __ffma2_rn(make_float2(cd, cd), make_float2(x[2 * h], x[2 * h + 1]),
                                                                      acc2[ADJ ? t : 0][h]);
                            }
                        }
                    }
                    // a stage that any thread gave up on stops the unit: nothing more is issued and
                    // the stage stays owed (n_used not advanced) for the bounded drain below
                    if (csync_or(tmo)) {
                        aborted = 1;
                        break;
                    }
                    ++n_used;
                    if (s + NS < nst) {
                        if (warp == (s + NS) % nwarp) issue(s + NS, n_issued);
                        ++n_issued;
                    }
                }
                if (tid == 0) s_pipe = aborted || (ld_volatile(L.err) == ERR_PIPE);
                csync();
                if (s_pipe) {
                    if (tid == 0) {
                        const long long t0 = globaltimer();
                        while (n_used < n_issued && globaltimer() - t0 < L.timeout_ns) {
                            const int bb = (int)(n_used % (uint32_t)NS);
                            if (mbar_try_wait(&bars[bb], (n_used / (uint32_t)NS) & 1u)) ++n_used;
                        }
                    }
                    break;
                }
                // With block-long update units, a running sum over the tile's chunks in chunk order:
                // chunk c stores S_c = S_{c-1} + p_c (S_{-1} = 0), the same adds, in the same order,
                // as a sequential sum of the C partials, and the update unit reads S_{C-1} alone
                // (its setup is on the step-to-step chain).  Chunk c-1 was claimed earlier, so the
                // wait ends; the tile's count says how many chunks are summed.  Per-step update
                // units sum the C partials themselves: their many short chunks run side by side,
                // where a chain of adds would serialise them.
                const int c0 = U.chunk;
                const bool chain = I.ub && c0 > 0;
                if (chain) {
                    if (tid == 0) {
                        const int w = wait_until(&I.arrive[par * I.T + tile], arrive_target(b, c0), L, 512);
                        if (w < 0) note_failure(L, 10, b, tile, arrive_target(b, c0), ld_acquire(&I.arrive[par * I.T + tile]), L.k0, 0);
                        s_ok = w > 0;
                    }
                    csync();
                    if (!s_ok) break;
                }
                if (j0 < I.N) {
                    auto add_store = [&](int t, int pl, float a0, float a1, float a2, float a3) {
                        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (chain) sum = __ldcg(reinterpret_cast<const float4 *>(prow(c0 - 1, t, pl) + j0));
                        sum.x += a0;
                        sum.y += a1;
                        sum.z += a2;
                        sum.w += a3;
                        *reinterpret_cast<float4 *>(prow(c0, t, pl) + j0) = sum;
                    };
    #pragma unroll
                    for (int t = 0; t < TB; ++t) {
                        add_store(t, 0, acc[t][0].x, acc[t][0].y, acc[t][1].x, acc[t][1].y);
                        if (ADJ)
                            add_store(t, 1, acc2[ADJ ? t : 0][0].x, acc2[ADJ ? t : 0][0].y, acc2[ADJ ? t : 0][1].x,
                                      acc2[ADJ ? t : 0][1].y);
                    }
                }
                // CTA barrier, then one release add: cumulative over every thread's partial stores
                csync();
                if (tid == 0) atom_add_acq_rel(&I.arrive[par * I.T + tile], 1u);
                continue;
            }
        }

        const float S = (float)I.S, dt = (float)I.dt;
        const float q0 = (float)I.react[0], q1 = (float)I.react[1], q2 = (float)I.react[2],
                    q3 = (float)I.react[3];
        const float *psi = reinterpret_cast<const float *>(I.psi);
        const float *dpsi = reinterpret_cast<const float *>(I.dpsi);
        const bool mirror = (I.bc == 1);
        const int kend = min(L.k_end, I.ksteps);
        // Rows of the newest 2T steps in FP32: the history itself for FP32 history, else the ring
        // of FP32 rows kept beside the low-precision history (row r in slot r mod hring_cap).
        auto hrow_at = [&](int r) -> const float * {
            return reinterpret_cast<const float *>(I.hring + (size_t)(r % I.hring_cap) * I.hring_pitch) + j0;
        };
        // Four values of history row r (any age) converted to FP32, FP16 scale applied (paired
        // history: hi + lo).
        auto hist4 = [&](int r) -> float4 {
            float x[4];
            if constexpr (PAIR) {
                const char *row = I.hist + (size_t)(r % I.cap) * I.pitch + (size_t)j0 * 2;
                float xl[4];
                H4<__half>::ldg(row, x);
                H4<__half>::ldg(row + (size_t)I.cap * I.pitch, xl);
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] += xl[v];
            } else {
                H4<TH>::ldg(I.hist + (size_t)(r % I.cap) * I.pitch + (size_t)j0 * sizeof(TH), x);
            }
            if (SCALED) {
                const float sc = __ldcg(I.hscale + (size_t)(r % I.cap) * I.T + tile);
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] *= sc;
            }
            return make_float4(x[0], x[1], x[2], x[3]);
        };

        // Phase B of step k on this tile: wait for u^k on the halo tiles, optionally add lag 1
        // (row k-1), apply the stencil, the reaction and the update (eq. frac_final; adjoint: the
        // reverse-time recursion), append delta^k and publish the tile's step.  H/H2 hold the rest
        // of the memory sum; d receives delta^k.  False when a wait gave up.
        // With own != null (block-long units) the tile's own u^k and low parts come from the
        // unit itself: own[0..V) and own[V..2V) in registers, and us[P] in shared memory for the
        // stencil's in-tile neighbours (us_next receives u^{k+1}); only halo points are loaded.
        int t0p = tile * I.P;  // first point of the tile
        auto phase_b = [&](int k, bool add_lag1, float *H, float *H2, float *d, bool last, float *own,
                           const float *us, float *us_next) -> bool {
            const int rel = k - L.k0;
            if (tid < 32) {  // one lane per halo tile
                int ok = 1;
                const int h = (I.ndim == 3) ? I.nx * I.ny : (I.ndim == 2) ? I.nx : 1;
                const int lo = max(0, tile * I.P - h) / I.P;
                const int hi = min(I.N - 1, tile * I.P + I.P - 1 + h) / I.P;
                for (int tt = lo + tid; tt <= hi && ok; tt += 32)
                    if (rel > 0) {
                        const int w = wait_until(&I.done[tt], (unsigned)rel, L, 32);
                        if (w < 0) note_failure(L, 5, k, tile, tt, rel, ld_acquire(&I.done[tt]), L.k0);
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
            csync();
            if (!s_ok2) return false;
            const float *uk = reinterpret_cast<const float *>(I.ubuf[k & 1]);
            float *un = reinterpret_cast<float *>(I.ubuf[(k + 1) & 1]);
            const float *lo_k = I.ulo[0] ? reinterpret_cast<const float *>(I.ulo[k & 1]) : nullptr;
            float *lo_n = I.ulo[0] ? reinterpret_cast<float *>(I.ulo[(k + 1) & 1]) : nullptr;
            const bool tape_row = I.tape && (k + 1 - I.tape_k0) >= 0 && ((k + 1 - I.tape_k0) % I.tape_every) == 0 &&
                                  ((k + 1 - I.tape_k0) / I.tape_every) < I.tape_rows;
            float *tp = tape_row ? reinterpret_cast<float *>(I.tape) + (size_t)((k + 1 - I.tape_k0) / I.tape_every) * I.N
                                 : nullptr;
            bool bad = false;
            double dl[6] = {0, 0, 0, 0, 0, 0};
            const float *ua = nullptr;
            if (ADJ) ua = reinterpret_cast<const float *>(I.uadj) + (size_t)((I.adj_K - 1 - k) - I.uadj_r0) * I.N;
#pragma unroll
            for (int v = 0; v < V; ++v) d[v] = 0.f;
            if (j0 < I.N) {
                // Every operand of the update is loaded before any is used, so that the loads of
                // this step's critical path are in flight together: row k-1, u^k and its
                // neighbours, the state's low part and (adjoint) u^r.
                const float4 x1 = add_lag1 ? __ldcg(reinterpret_cast<const float4 *>(hrow_at(k - 1)))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                const int pl = I.nx * I.ny;
                float cu[V], nb[V][6], lw[V], ur[V];
                unsigned inb[V];  // bit e: neighbour e inside the grid (r, l, up, dn, fw, bk)
                // a point inside this tile comes from shared memory when the unit keeps it
                auto get1 = [&](int jn) -> float {
                    return (own && jn >= t0p && jn < t0p + I.P) ? us[jn - t0p] : __ldcg(uk + jn);
                };
                // four consecutive points from jn (a multiple of 4), in one 16-byte load
                auto get4 = [&](int jn, float *o) {
                    float4 w;
                    if (own && jn >= t0p && jn + 3 < t0p + I.P)
                        w = *reinterpret_cast<const float4 *>(us + (jn - t0p));
                    else
                        w = __ldcg(reinterpret_cast<const float4 *>(uk + jn));
                    o[0] = w.x;
                    o[1] = w.y;
                    o[2] = w.z;
                    o[3] = w.w;
                };
                grid_masks<V>(I, j0, inb);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = j0 + v;
                    const bool in = j < I.N;
#pragma unroll
                    for (int e = 0; e < 6; ++e) nb[v][e] = 0.f;
                    lw[v] = (!in || !lo_k) ? 0.f : own ? own[V + v] : __ldcg(lo_k + j);
                    ur[v] = (ADJ && in) ? __ldcg(ua + j) : 0.f;
                }
                if (j0 + V <= I.N) {
                    // all four points in the grid: the centre in one load, x-neighbours inside
                    // the vector from it (a set mask bit means the same row), y/z-neighbours in
                    // one load each where the row (plane) length keeps them aligned
                    if (own) {
#pragma unroll
                        for (int v = 0; v < V; ++v) cu[v] = own[v];
                    } else {
                        get4(j0, cu);
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (inb[v] & 1u) nb[v][0] = (v + 1 < V) ? cu[v + 1] : get1(j0 + V);
                        if (inb[v] & 2u) nb[v][1] = (v > 0) ? cu[v - 1] : get1(j0 - 1);
                    }
                    auto vert = [&](int e, unsigned bit, int off, int len) {
                        if ((len & 3) == 0) {  // the four share a row (plane): one mask for all
                            if (inb[0] & bit) {
                                float o[V];
                                get4(j0 + off, o);
#pragma unroll
                                for (int v = 0; v < V; ++v) nb[v][e] = o[v];
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (inb[v] & bit) nb[v][e] = get1(j0 + v + off);
                        }
                    };
                    if (I.ndim >= 2) {
                        vert(2, 4u, I.nx, I.nx);
                        vert(3, 8u, -I.nx, I.nx);
                    }
                    if (I.ndim == 3) {
                        vert(4, 16u, pl, pl);
                        vert(5, 32u, -pl, pl);
                    }
                } else {  // the grid's ragged end: point by point
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int j = j0 + v;
                        const unsigned m = inb[v];
                        cu[v] = (j >= I.N) ? 0.f : own ? own[v] : __ldcg(uk + j);
                        if (m & 1u) nb[v][0] = get1(j + 1);
                        if (m & 2u) nb[v][1] = get1(j - 1);
                        if (m & 4u) nb[v][2] = get1(j + I.nx);
                        if (m & 8u) nb[v][3] = get1(j - I.nx);
                        if (m & 16u) nb[v][4] = get1(j + pl);
                        if (m & 32u) nb[v][5] = get1(j - pl);
                    }
                }
                if (ADJ) adjoint_tail<float, float, V>(I, k, j0, H, H2);
                if (add_lag1) {  // lag 1 completes the memory sum
                    const float cc = psi[1];
                    H[0] = fmaf(cc, x1.x, H[0]);
                    H[1] = fmaf(cc, x1.y, H[1]);
                    H[2] = fmaf(cc, x1.z, H[2]);
                    H[3] = fmaf(cc, x1.w, H[3]);
                    if (ADJ) {
                        const float c2 = dpsi[1];
                        H2[0] = fmaf(c2, x1.x, H2[0]);
                        H2[1] = fmaf(c2, x1.y, H2[1]);
                        H2[2] = fmaf(c2, x1.z, H2[2]);
                        H2[3] = fmaf(c2, x1.w, H2[3]);
                    }
                }
                float nvv[V], nlv[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = j0 + v;
                    nvv[v] = cu[v];
                    nlv[v] = 0.f;
                    if (j >= I.N) continue;
                    const float c = cu[v];
                    const float gh = mirror ? c : 0.f;
                    const unsigned m = inb[v];
                    const float r = (m & 1u) ? nb[v][0] : gh, l = (m & 2u) ? nb[v][1] : gh;
                    if (I.ndim == 1) {
                        d[v] = r - 2.f * c + l;
                    } else {
                        const float up = (m & 4u) ? nb[v][2] : gh, dn = (m & 8u) ? nb[v][3] : gh;
                        if (I.ndim == 2) {
                            d[v] = r + l - 4.f * c + up + dn;
                        } else {
                            const float fw = (m & 16u) ? nb[v][4] : gh, bk = (m & 32u) ? nb[v][5] : gh;
                            d[v] = r + l - 6.f * c + up + dn + fw + bk;
                        }
                    }
                    const float G = d[v] + H[v];  // psi_0 times the fresh row plus the memory sum
                    float inc;
                    if (!ADJ) {
                        const float f = q0 + c * (q1 + c * (q2 + c * q3));
                        inc = dt * f + S * G;
                    } else {
                        // reverse-time recursion: lambda^r = lambda^{r+1} + dt f'(u^r) lambda^{r+1} + S G
                        const float u_r = ur[v];
                        const float fp = q1 + u_r * (2.f * q2 + u_r * 3.f * q3);
                        inc = dt * fp * c + S * G;
                        dl[0] += (double)u_r * (double)G;
                        dl[1] += (double)u_r * (double)H2[v];
                        double pw = 1.0;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            dl[2 + i] += (double)c * pw;
                            pw *= (double)u_r;
                        }
                    }
                    float nl = 0.f;
                    if (lo_k) {
                        const float y2 = inc + lw[v];
                        const float sum = c + y2;
                        const float bb = sum - c;
                        nl = (c - (sum - bb)) + (y2 - bb);
                        nvv[v] = sum;
                    } else {
                        nvv[v] = c + inc;
                    }
                    nlv[v] = nl;
                    bad |= !isfinite(nvv[v]);
                }
                // stores: 16-byte vectors where all four points exist
                if (j0 + V <= I.N) {
                    *reinterpret_cast<float4 *>(un + j0) = make_float4(nvv[0], nvv[1], nvv[2], nvv[3]);
                    if (lo_n) *reinterpret_cast<float4 *>(lo_n + j0) = make_float4(nlv[0], nlv[1], nlv[2], nlv[3]);
                    if (own)
                        *reinterpret_cast<float4 *>(us_next + (j0 - t0p)) = make_float4(nvv[0], nvv[1], nvv[2], nvv[3]);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (j0 + v < I.N) {
                            un[j0 + v] = nvv[v];
                            if (lo_n) lo_n[j0 + v] = nlv[v];
                            if (own) us_next[j0 + v - t0p] = nvv[v];
                        }
                }
                if (tp) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (j0 + v < I.N) tp[j0 + v] = nvv[v];
                }
                if (own) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        own[v] = nvv[v];
                        own[V + v] = nlv[v];
                    }
                }
                if (I.hist_write) {
                    // delta^k in FP32 for the near lags (for FP32 history, the history row itself)
                    *reinterpret_cast<float4 *>(I.hring + (size_t)(k % I.hring_cap) * I.hring_pitch + (size_t)j0 * 4) =
                        make_float4(d[0], d[1], d[2], d[3]);
                    if (LOWP && !F16) {
                        char *row = I.hist + (size_t)(k % I.cap) * I.pitch + (size_t)j0 * sizeof(TH);
                        H4<TH>::stg(row, d, 1.f);
                        if (TC && I.lo_plane) {  // the rounding remainder, for tensor-core near/mid units
                            float dr[V];
#pragma unroll
                            for (int v = 0; v < V; ++v) dr[v] = d[v] - __bfloat162float(__float2bfloat16_rn(d[v]));
                            H4<TH>::stg(row + (size_t)I.cap * I.pitch, dr, 1.f);
                        }
                    }
                }
            }
            if (SCALED && I.hist_write) {
                // FP16 row (or FP32 row as an FP16 hi/lo pair): a power-of-two scale per (row,
                // tile) from the tile's largest |delta|
                float amax = 0.f;
#pragma unroll
                for (int v = 0; v < V; ++v) amax = fmaxf(amax, fabsf(d[v]));  // zero past the grid's end
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                if ((tid & 31) == 0) s_wmax[tid >> 5] = amax;
                csync();
                float m = 0.f;
                for (int w = 0; w < (nthr + 31) / 32; ++w) m = fmaxf(m, s_wmax[w]);
                int e = 0;
                if (m > 0.f && isfinite(m)) {
                    int ex;
                    frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
                    e = max(-100, min(100, 15 - ex));
                }
                if (tid == 0) I.hscale[(size_t)(k % I.cap) * I.T + tile] = ldexpf(1.f, -e);
                if (j0 < I.N) {
                    const float sc = ldexpf(1.f, e);
                    char *row = I.hist + (size_t)(k % I.cap) * I.pitch + (size_t)j0 * 2;
                    if (F16) {
                        H4<__half>::stg(row, d, sc);
                        if (TC && I.lo_plane) {  // the rounding remainder, for tensor-core near/mid units
                            float dr[V];
#pragma unroll
                            for (int v = 0; v < V; ++v) dr[v] = d[v] * sc - __half2float(__float2half_rn(d[v] * sc));
                            H4<__half>::stg(row + (size_t)I.cap * I.pitch, dr, 1.f);
                        }
                    } else {  // paired: hi = fp16(d 2^e), lo = fp16(d 2^e - hi), both exact scalings
                        float dh[V], dr[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            dh[v] = __half2float(__float2half_rn(d[v] * sc));
                            dr[v] = d[v] * sc - dh[v];
                        }
                        H4<__half>::stg(row, dh, 1.f);
                        H4<__half>::stg(row + (size_t)I.cap * I.pitch, dr, 1.f);
                    }
                }
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
            // History rows are read later by bulk copies (async proxy): order this thread's
            // generic stores before them, then publish with one release after the CTA barrier.
            // A block-long unit fences once, at its last step: bulk copies read a block's rows
            // only after that step's release, and the fence covers all of the thread's earlier
            // stores.
            if (!own || last) fence_proxy_async_global();
            csync();
            if (tid == 0) {
                if (ADJ) {  // per-tile gradient partials, one writer per tile, in step order
                    double *dd = I.dots + (size_t)tile * 8;
                    for (int i = 0; i < 6; ++i) {
                        double sacc = 0.0;
                        for (int w = 0; w < (nthr + 31) / 32; ++w) sacc += s_dred[w][i];
                        dd[i] += sacc;
                    }
                }
                // the block's last update for this tile sets the far count word for block
                // b+npar, whose far units wait for this step before they count
                if (last) I.arrive[par * I.T + tile] = arrive_target(b + I.npar, 0);
                st_release(&I.done[tile], (unsigned)(rel + 1));
            }
            return true;
        };

        if (U.fix == 3 || U.fix == 4) {
            // ======================= near unit: the previous block's rows for every step of block b
            // N_t = sum over rows r = kb-TB .. kb-1 (oldest first) of w_{kb+t}(kb+t-r) delta^r, from
            // the FP32 rows: psi (short memory: 0 beyond the window; adaptive memory: the settled
            // weight g(m) up to the step's e(k), psi beyond).  Written as partial row C of block b
            // and counted like a far chunk, so each step's update reads one row for these lags
            // instead of TB.  The weights are staged in the idle stage ring.
            // Mid unit (fix 4): the same sum over the block's own rows kb .. kb+s-1 for the steps
            // t = s .. s+15 of sub-block s/16, written as partial row C+1; an update then reads at
            // most 15 head rows, those of its own sub-block.
            const int t_lo = (U.fix == 4) ? U.k - kb : 0, t_hi = (U.fix == 4) ? t_lo + 16 : TB;
            const int r0 = U.r0, r1 = U.r1, mlo = kb + t_lo - r1 + 1;  // smallest lag
            float *spsi = reinterpret_cast<float *>(stages), *sgw = spsi + 2 * TB;
            const float *gwf = reinterpret_cast<const float *>(I.gw);
            for (int e = tid; e < 2 * TB; e += nthr) {
                const int m = mlo + e;
                const float c = (I.mem_mode == 1 && m > I.mem_L) ? 0.f : psi[m];
                spsi[e] = c;
                sgw[e] = gwf ? gwf[m] : c;
            }
            if (tid < TB) s_ek[tid] = (gwf && kb + tid < I.ksteps) ? settled_end(I, kb + tid) : 0x7fffffff;
            csync();
            constexpr int TG = TB < 8 ? TB : 8;  // steps per pass (register budget: no spills)
            for (int tg = t_lo; tg < t_hi; tg += TG) {
                float2 acc[TG][2];
#pragma unroll
                for (int t = 0; t < TG; ++t) acc[t][0] = acc[t][1] = make_float2(0.f, 0.f);
                for (int r = r0; r < r1; r += 8) {
                    float4 x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        x[i] = (r + i < r1 && j0 < I.N) ? __ldcg(reinterpret_cast<const float4 *>(hrow_at(r + i)))
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (r + i >= r1) continue;
#pragma unroll
                        for (int t = 0; t < TG; ++t) {
                            const int m = kb + tg + t - (r + i);
                            const float c = (gwf && m <= s_ek[tg + t]) ? sgw[m - mlo] : spsi[m - mlo];
                            const float2 c2 = make_float2(c, c);
                            acc[t][0] = __ffma2_rn(c2, make_float2(x[i].x, x[i].y), acc[t][0]);
                            acc[t][1] = __ffma2_rn(c2, make_float2(x[i].z, x[i].w), acc[t][1]);
                        }
                    }
                }
                if (j0 < I.N) {
#pragma unroll
                    for (int t = 0; t < TG; ++t)
                        if (kb + tg + t < I.ksteps)
                            *reinterpret_cast<float4 *>(prow(U.chunk, tg + t, 0) + j0) =
                                make_float4(acc[t][0].x, acc[t][0].y, acc[t][1].x, acc[t][1].y);
                }
            }
            // the ring is filled by bulk copies again: order this thread's accesses before them;
            // then a CTA barrier and one release add, as for a far chunk
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            csync();
            if (tid == 0) atom_add_acq_rel(&I.arrive[par * I.T + tile], 1u);
            continue;
        }

        if constexpr (!TC) if (U.fix == 2) {
            // ============================ block-long update unit: every step of block b, this tile
            // The block's steps run in order on this CTA.  The memory sum of step kb+t is the
            // running sum of the block's far chunks, then (adaptive memory) the tail rows below
            // the far rows, then the rows before the block (read once, oldest first), then the
            // rows of the block's earlier steps, which this unit produced itself: each new
            // delta^k is folded into the sums of the later steps right after its update.  The
            // summation order per step is that of the per-step units (partials by chunk, then
            // rows by increasing row index), so results agree with them to the bit when the
            // chunks agree.  The sums live in the stage ring, idle during this unit.
            const int kf = max(kb, L.k0), kl = min(kb + TB, kend);
            if (tid < TB) s_ek[tid] = (I.gw && kb + tid < I.ksteps) ? settled_end(I, kb + tid) : 0x7fffffff;
            if (tid < 32) {
                int ok = 1;
                if (tid == 0) {
                    const int w = wait_until(&I.arrive[par * I.T + tile], arrive_target(b, C), L, 512);
                    if (w < 0) note_failure(L, 3, kf, tile, arrive_target(b, C), ld_acquire(&I.arrive[par * I.T + tile]), L.k0, 0);
                    ok = w > 0;
                }
                if (tid == 1 && kf - L.k0 > 0) {  // this tile's rows up to kf-1
                    const int w = wait_until(&I.done[tile], (unsigned)(kf - L.k0), L, 512);
                    if (w < 0) note_failure(L, 4, kf, tile, kf - L.k0, ld_acquire(&I.done[tile]), L.k0, 0);
                    ok = w > 0;
                }
                ok = __all_sync(0xffffffffu, ok);
                if (tid == 0) s_ok = ok;
            }
            csync();
            if (!s_ok) break;
            float4 *Hs = reinterpret_cast<float4 *>(stages);  // [TB][nthr] sums of the block's steps
            float4 *Hs2 = Hs + TB * nthr;                      // psi' sums (adjoint)
            const int t0 = kf - kb, t1 = kl - kb;
            auto window = [&](int k) { return (I.mem_mode == 1) ? min(I.mem_L, k) : k; };
            if (j0 < I.N) {
                // Far part of every step from the running sum, then the rows before kf (the
                // previous block's and, when this launch starts inside the block, the block's
                // earlier ones), oldest first.  The sums stay in registers and each group of
                // loads is in flight together: this setup is on the step-to-step chain.
                float4 h[TB], h2[ADJ ? TB : 1];
#pragma unroll
                for (int t = 0; t < TB; ++t) {
                    h[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ADJ) h2[ADJ ? t : 0] = h[t];
                    if (C > 0 && t >= t0 && t < t1) {
                        h[t] = __ldcg(reinterpret_cast<const float4 *>(prow(C - 1, t, 0) + j0));
                        if (ADJ) h2[ADJ ? t : 0] = __ldcg(reinterpret_cast<const float4 *>(prow(C - 1, t, 1) + j0));
                    }
                }
                // rows [ra, rb) with each step's weight of their lag, four loads in flight
                const float *gwf = reinterpret_cast<const float *>(I.gw);
                // (old: tail rows from the history of any age; else the near rows in FP32)
                auto add_rows = [&](int ra, int rb, bool old) {
                    for (int r = ra; r < rb; r += 4) {
                        float4 x[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            x[i] = (r + i >= rb) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : old         ? hist4(r + i)
                                                 : __ldcg(reinterpret_cast<const float4 *>(hrow_at(r + i)));
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int t = 0; t < TB; ++t) {
                                const int lag = kb + t - (r + i);
                                if (r + i >= rb || t < t0 || t >= t1 || lag > window(kb + t)) continue;
                                const float cc = (I.gw && lag <= s_ek[t]) ? gwf[lag] : psi[lag];
                                h[t].x = fmaf(cc, x[i].x, h[t].x);
                                h[t].y = fmaf(cc, x[i].y, h[t].y);
                                h[t].z = fmaf(cc, x[i].z, h[t].z);
                                h[t].w = fmaf(cc, x[i].w, h[t].w);
                                if (ADJ) {
                                    const float c2 = dpsi[lag];
                                    float4 &g = h2[ADJ ? t : 0];
                                    g.x = fmaf(c2, x[i].x, g.x);
                                    g.y = fmaf(c2, x[i].y, g.y);
                                    g.z = fmaf(c2, x[i].z, g.z);
                                    g.w = fmaf(c2, x[i].w, g.w);
                                }
                            }
                    }
                };
                if (I.gw) {  // adaptive memory: the tail rows below the far rows
                    int rlo, rhi;
                    far_rows<TB>(I, b, rlo, rhi);
                    add_rows(0, rlo, true);
                }
                add_rows(max(0, kb - TB), kf, false);
#pragma unroll
                for (int t = 0; t < TB; ++t)
                    if (t >= t0 && t < t1) {
                        Hs[t * nthr + tid] = h[t];
                        if (ADJ) Hs2[t * nthr + tid] = h2[ADJ ? t : 0];
                    }
            }
            // the tile's own u^kf and low parts: registers, and u in shared memory for the stencil
            float own[2 * V];
            float *us = reinterpret_cast<float *>(Hs + TB * PLANES * nthr);  // [2][P]: u^k by k parity
            {
                const float *u0 = reinterpret_cast<const float *>(I.ubuf[kf & 1]);
                const float *l0 = I.ulo[0] ? reinterpret_cast<const float *>(I.ulo[kf & 1]) : nullptr;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = j0 + v;
                    own[v] = (j < I.N) ? __ldcg(u0 + j) : 0.f;
                    own[V + v] = (j < I.N && l0) ? __ldcg(l0 + j) : 0.f;
                    if (j < I.N) us[(kf & 1) * I.P + (j - t0p)] = own[v];
                }
            }
            csync();
            bool stop = false;
            for (int t = t0; t < t1; ++t) {
                const int k = kb + t;
                float H[V], H2[V], d[V];
                const float4 h = (j0 < I.N) ? Hs[t * nthr + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 h2 = (ADJ && j0 < I.N) ? Hs2[t * nthr + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
                H[0] = h.x;
                H[1] = h.y;
                H[2] = h.z;
                H[3] = h.w;
                H2[0] = h2.x;
                H2[1] = h2.y;
                H2[2] = h2.z;
                H2[3] = h2.w;
                if (!phase_b(k, false, H, H2, d, k == kl - 1, own, us + (k & 1) * I.P, us + ((k + 1) & 1) * I.P)) {
                    stop = true;
                    break;
                }
                if (j0 < I.N) {  // delta^k enters the later steps of the block
                    for (int t2 = t + 1; t2 < t1; ++t2) {
                        const int lag = t2 - t;
                        if (lag > window(kb + t2)) continue;
                        const float cc = (I.gw && lag <= s_ek[t2]) ? reinterpret_cast<const float *>(I.gw)[lag] : psi[lag];
                        float4 a = Hs[t2 * nthr + tid];
                        a.x = fmaf(cc, d[0], a.x);
                        a.y = fmaf(cc, d[1], a.y);
                        a.z = fmaf(cc, d[2], a.z);
                        a.w = fmaf(cc, d[3], a.w);
                        Hs[t2 * nthr + tid] = a;
                        if (ADJ) {
                            const float c2 = dpsi[lag];
                            float4 a2 = Hs2[t2 * nthr + tid];
                            a2.x = fmaf(c2, d[0], a2.x);
                            a2.y = fmaf(c2, d[1], a2.y);
                            a2.z = fmaf(c2, d[2], a2.z);
                            a2.w = fmaf(c2, d[3], a2.w);
                            Hs2[t2 * nthr + tid] = a2;
                        }
                    }
                }
            }
            if (stop) break;
            // the ring is filled by bulk copies again: order this thread's accesses before them
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            continue;
        }

        // ================================================== update unit: step k, tiles U.tile ..
        // (tensor-core kernels: I.ug consecutive tiles per unit, so that a step has fewer units than
        // the grid has half-CTAs and each unit's claim and waits are paid once for its tiles)
        const int k = U.k, t = k - kb;
        const int rel = k - L.k0;
        const int nmid = I.mid ? min(I.mid, t / 16) : 0;  // mid units of sub-blocks 1 .. t/16
        const int ntl = min(I.ug, I.T - U.tile);          // tiles of this unit
        // Two phases keep the partial and head sums off the step-to-step chain.  Phase A needs
        // only the tile's far count and this tile's rows up to k-2 (its own step k-2), so it
        // runs while step k-1 is still being updated; phase B waits for u^k on the halo tiles
        // and row k-1, then adds lag 1 and updates.  The summation order is unchanged:
        // partials by chunk, then lags hk .. 1.
        if (tid < 32) {  // the waits run in parallel lanes: far counts in lanes 0.., own rows in 16..
            int ok = 1;
            const unsigned tgt = arrive_target(b, C * L.fsub + (I.near + nmid) * nsub);
            if (tid < ntl) {  // the far chunks and, with near units, the near (and mid) partials
                const int tt = U.tile + tid;
                const int w = wait_until(&I.arrive[par * I.T + tt], tgt, L, 512);
                if (w < 0) note_failure(L, 3, k, tt, tgt, ld_acquire(&I.arrive[par * I.T + tt]), L.k0, 0);
                ok = w > 0;
            }
            if (tid >= 16 && tid < 16 + ntl && rel > 1) {
                const int tt = U.tile + tid - 16;
                const int w = wait_until(&I.done[tt], (unsigned)(rel - 1), L, 512);
                if (w < 0) note_failure(L, 4, k, tt, rel - 1, ld_acquire(&I.done[tt]), L.k0, 0);
                ok = w > 0;
            }
            ok = __all_sync(0xffffffffu, ok);
            if (tid == 0) s_ok = ok;
        }
        csync();
        if (!s_ok) break;

        const int nb = (I.mem_mode == 1) ? min(I.mem_L, k) : k;
        // head: lags 1 .. min(k-kb+T, n_base(k)), descending; with a near unit only the block's
        // own rows, lags 1 .. min(k-kb, n_base(k)) (the near partial holds the previous block's)
        const int hk = I.near ? min(I.mid ? t % 16 : t, nb) : min(t + TB, nb);
        const int CP = C + I.near + (nmid ? 1 : 0);  // partial rows to sum
        auto hrow = [&](int m) -> const float * { return hrow_at(k - m); };
        constexpr int UG = TC ? 2 : 1;  // most tiles per update unit
        float HG[UG][V], H2G[UG][V], d[V];
#pragma unroll
        for (int g = 0; g < UG; ++g) {  // phase A of each tile
            if (g >= ntl) break;
            tile = U.tile + g;
            j0 = tile * I.P + tid * V;
            t0p = tile * I.P;
            float *H = HG[g], *H2 = H2G[g];
#pragma unroll
            for (int v = 0; v < V; ++v) H[v] = H2[v] = 0.f;
            if (j0 < I.N) {
                // far part: chunk partials in fixed order, G loads in flight (the unit is latency-bound:
                // its loads are all it does before the halo wait)
                // Batches of G rows whose last one re-reads a valid row in place of the missing
                // ones and leaves them out of the sums, so that every load of a batch is in flight
                // together: a step has about one batch of partial rows and up to two of head rows,
                // and a partial batch must not fall back to one row per round trip.
                constexpr int G = ADJ ? 4 : 8;
                for (int c = 0; c < CP; c += G) {
                    float4 w[G], w2[ADJ ? G : 1];
    #pragma unroll
                    for (int i = 0; i < G; ++i) {
                        const int ci = min(c + i, CP - 1);
                        w[i] = __ldcg(reinterpret_cast<const float4 *>(prow(ci, t, 0) + j0));
                        if (ADJ) w2[ADJ ? i : 0] = __ldcg(reinterpret_cast<const float4 *>(prow(ci, t, 1) + j0));
                    }
    #pragma unroll
                    for (int i = 0; i < G; ++i) {
                        if (c + i >= CP) continue;
                        H[0] += w[i].x;
                        H[1] += w[i].y;
                        H[2] += w[i].z;
                        H[3] += w[i].w;
                        if (ADJ) {
                            H2[0] += w2[ADJ ? i : 0].x;
                            H2[1] += w2[ADJ ? i : 0].y;
                            H2[2] += w2[ADJ ? i : 0].z;
                            H2[3] += w2[ADJ ? i : 0].w;
                        }
                    }
                }
                // weight of lag m at this step (adaptive memory: settled or tail weight)
                const int ek = I.gw ? settled_end(I, k) : 0x7fffffff;
                auto wgt = [&](int m) -> float {
                    return (I.gw && m <= ek) ? reinterpret_cast<const float *>(I.gw)[m] : psi[m];
                };
                if (!ADJ && I.gw) {
                    // adaptive memory: the tail rows below the far rows, oldest first
                    int rlo, rhi;
                    far_rows<TB>(I, b, rlo, rhi);
                    for (int r = 0; r < rlo; r += 4) {
                        float4 x[4];
    #pragma unroll
                        for (int i = 0; i < 4; ++i) x[i] = (r + i < rlo) ? hist4(r + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    #pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (r + i >= rlo) continue;
                            const float cc = wgt(k - (r + i));
                            H[0] = fmaf(cc, x[i].x, H[0]);
                            H[1] = fmaf(cc, x[i].y, H[1]);
                            H[2] = fmaf(cc, x[i].z, H[2]);
                            H[3] = fmaf(cc, x[i].w, H[3]);
                        }
                    }
                }
                // head lags hk .. 2: rows this tile wrote at steps up to k-2, G loads in flight
                for (int m = hk; m >= 2; m -= G) {
                    float4 x[G];
    #pragma unroll
                    for (int i = 0; i < G; ++i) x[i] = __ldcg(reinterpret_cast<const float4 *>(hrow(max(m - i, 2))));
    #pragma unroll
                    for (int i = 0; i < G; ++i) {
                        if (m - i < 2) continue;
                        const float cc = wgt(m - i);
                        H[0] = fmaf(cc, x[i].x, H[0]);
                        H[1] = fmaf(cc, x[i].y, H[1]);
                        H[2] = fmaf(cc, x[i].z, H[2]);
                        H[3] = fmaf(cc, x[i].w, H[3]);
                        if (ADJ) {
                            const float c2 = dpsi[m - i];
                            H2[0] = fmaf(c2, x[i].x, H2[0]);
                            H2[1] = fmaf(c2, x[i].y, H2[1]);
                            H2[2] = fmaf(c2, x[i].z, H2[2]);
                            H2[3] = fmaf(c2, x[i].w, H2[3]);
                        }
                    }
                }
            }
        }
        bool units_ok = true;
#pragma unroll
        for (int g = 0; g < UG; ++g) {  // phase B of each tile, in tile order
            if (g >= ntl) break;
            tile = U.tile + g;
            j0 = tile * I.P + tid * V;
            t0p = tile * I.P;
            if (!phase_b(k, hk >= 1, HG[g], H2G[g], d, k == min(kb + TB, kend) - 1, nullptr, nullptr, nullptr)) {
                units_ok = false;
                break;
            }
        }
        if (!units_ok) break;
    }
    // every exit from the unit loop is CTA-uniform; the tensor memory goes back once all of the
    // CTA's tensor-core work has completed (a failed unit waits for its MMAs before it exits)
    if (TC) {
        tc::fence_before();
        __syncthreads();  // both halves
        if (threadIdx.x < 32) {
            tc::fence_after();
            tc::tmem_dealloc(s_tmem, tc_cols * HALVES);
        }
    }
}

}  // namespace fdk

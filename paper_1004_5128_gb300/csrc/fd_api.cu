// fd_api.cu -- host runtime behind include/fd.h.
//
// Builds the GL weights (Section 2.1 recurrence) and the memory schedule of each
// step (eq. frac_final, eq. frac_shortmemory, Proposition 3.1) on the host in
// FP64/integers, lays out the caller's workspace, uploads the tables and drives
// the persistent engine (fd_engine.cuh): forward launches, the checkpointed
// reverse-time adjoint, and multi-instance batches recorded as a CUDA graph.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include <nvtx3/nvToolsExt.h>
#include <new>
#include <vector>

#include "../../include/fd.h"
#include "fd_kernels.h"

using fdk::Inst;
using fdk::Launch;

namespace {

constexpr size_t kAlign = 256;
// Partial-row parities: a tile's chunks may run up to npar-1 steps (blocks) ahead of its
// update.  The per-step kernel takes 8 (its chunks need rows at least head+1 steps old, so 8
// parities let them overlap every step the history allows); the blocked kernel 4 (its far units
// run one block ahead of the updates, and partials are T rows per chunk).
inline int npar_for(int tb) { return tb ? 4 : 8; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int dtype_size(int d)
{
    switch (d) {
    case FD_F64: return 8;
    case FD_F32: return 4;
    case FD_BF16:
    case FD_F16: return 2;
    default: return 0;
    }
}

// Bump allocator over the caller's workspace (base == nullptr: size only).
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(char *b) : base(b) {}
    char *take(size_t bytes)
    {
        off = align_up(off, kAlign);
        char *p = base ? base + off : nullptr;
        off += align_up(bytes, kAlign);
        return p;
    }
};

// ------------------------------------------------------------ weights, schedule

// psi(g,0) = 1, psi(g,m) = psi(g,m-1) (m-2+g)/m ; dpsi is its derivative in g.
void gl_weights(double g, int64_t n, double *psi, double *dpsi)
{
    psi[0] = 1.0;
    if (dpsi) dpsi[0] = 0.0;
    for (int64_t m = 1; m < n; ++m) {
        const double f = ((double)m - 2.0 + g) / (double)m;
        psi[m] = psi[m - 1] * f;
        if (dpsi) dpsi[m] = dpsi[m - 1] * f + psi[m - 1] / (double)m;
    }
}

struct Median {
    int lag, mult;
    int64_t end;  // last lag the increment stands for
};

// Adaptive medians in order of increment end, up to increments ending <= kmax.
std::vector<Median> adaptive_medians(int64_t a, int rule, int64_t kmax)
{
    std::vector<Median> G;
    if (a < 2) return G;
    if (rule == FD_ADAPT_PAPER) {
        // interval i >= 2: medians a^{i-1} + i + (eta-1)(2i-1) up to a^i, each standing for
        // lags m-(i-1) .. m+(i-1); intervals restart at a^{i-1}+1 whatever the previous end
        int64_t lo = a;  // a^{i-1}
        for (int64_t i = 2; lo + 1 <= kmax; ++i) {
            const int64_t hi = (lo > (int64_t)4e15 / a) ? (int64_t)4e15 : lo * a;
            const int64_t d = 2 * i - 1;
            for (int64_t m = lo + i; m <= hi; m += d) {
                if (m + i - 1 > kmax) return G;
                G.push_back({(int)m, (int)d, m + i - 1});
            }
            lo = hi;
        }
    } else {
        // a cursor tiles lags a+1.. with consecutive increments of width 2i-1
        int64_t c = a + 1, hi = a;
        for (int64_t i = 2;; ++i) {
            hi = (hi > (int64_t)4e15 / a) ? (int64_t)4e15 : hi * a;
            const int64_t d = 2 * i - 1;
            for (int64_t m = c + i - 1; m <= hi; m = c + i - 1) {
                if (c + d - 1 > kmax) return G;
                G.push_back({(int)m, (int)d, c + d - 1});
                c += d;
            }
        }
    }
    return G;
}

// Per-step device schedule (lags >= 1): nb base lags 1..nb, ng medians G[0..ng),
// tail lags tail_lo..tail_hi.
struct Sched {
    std::vector<int4> step;  // per k
    std::vector<Median> G;
};

int build_schedule(const fd_problem &p, int64_t K, Sched &s)
{
    s.step.resize(K);
    if (p.mem_mode == FD_MEM_ADAPTIVE) s.G = adaptive_medians(p.mem_a, p.adaptive_rule, K);
    size_t g = 0;
    for (int64_t k = 0; k < K; ++k) {
        int4 e = make_int4(0, 0, 1, 0);
        if (p.mem_mode == FD_MEM_FULL) {
            e.x = (int)k;
        } else if (p.mem_mode == FD_MEM_SHORT) {
            e.x = (int)std::min<int64_t>(p.mem_L, k);
        } else if (k <= p.mem_a) {
            e.x = (int)k;
        } else {
            e.x = p.mem_a;
            while (g < s.G.size() && s.G[g].end <= k) ++g;
            e.y = (int)g;
            const int64_t last = g ? s.G[g - 1].end : p.mem_a;
            e.z = (int)(last + 1);
            e.w = (int)k;
        }
        s.step[k] = e;
    }
    return FD_OK;
}

inline int64_t n_terms(const int4 &e) { return (int64_t)e.x + e.y + (e.w >= e.z ? e.w - e.z + 1 : 0); }

inline bool closed_loop(const fd_problem &p) { return (p.flags & FD_FLAG_CLOSED_LOOP) != 0; }

// The adjoint of adaptive memory runs the full-memory adjoint with the settled weights (plus the
// tail terms' corrections): its work units are those of full memory.
inline bool adaptive_adjoint(const fd_problem &p)
{
    return p.mem_mode == FD_MEM_ADAPTIVE && (p.flags & FD_FLAG_KEEP_TAPE);
}
inline fd_problem full_memory(const fd_problem &p)
{
    fd_problem q = p;
    q.mem_mode = FD_MEM_FULL;
    return q;
}
inline int4 full_step(int64_t k) { return make_int4((int)k, 0, 1, 0); }

// ------------------------------------------------------------------ validation

// Blocked runs multiply their far rows on the tensor cores with BF16 or FP16 history and blocks of
// 16, 32 or 64, and with FP32 history (as FP16 hi + lo planes) and blocks of 32 or 64, unless
// FD_FLAG_FMA_FAR asks for the CUDA-core loop; taped (adjoint) runs use the CUDA cores.
inline bool tc_far(const fd_problem &p)
{
    const bool lowp = (p.time_block == 16 || p.time_block == 32 || p.time_block == 64) &&
                      (p.hist_dtype == FD_BF16 || p.hist_dtype == FD_F16);
    const bool split = (p.time_block == 32 || p.time_block == 64) && p.hist_dtype == FD_F32;
    return (lowp || split) && !(p.flags & FD_FLAG_FMA_FAR) && !(p.flags & FD_FLAG_KEEP_TAPE);
}

int validate(const fd_problem *p)
{
    if (!p) return FD_ERR_INVALID_ARG;
    if (p->ndim < 1 || p->ndim > 3) return FD_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->ndim == 1 && p->ny != 1) || (p->ndim < 3 && p->nz != 1))
        return FD_ERR_INVALID_ARG;
    if ((int64_t)p->nx * p->ny * p->nz > (int64_t)1 << 30) return FD_ERR_INVALID_ARG;
    if (!(p->gamma > 0.0 && p->gamma < 2.0)) return FD_ERR_INVALID_ARG;
    if (!(p->alpha > 0.0) || !(p->dt > 0.0) || !(p->dx > 0.0)) return FD_ERR_INVALID_ARG;
    for (double r : p->react)
        if (!std::isfinite(r)) return FD_ERR_INVALID_ARG;
    if (p->bc != FD_BC_DIRICHLET0 && p->bc != FD_BC_NOFLUX) return FD_ERR_INVALID_ARG;
    if (p->mem_mode < FD_MEM_FULL || p->mem_mode > FD_MEM_ADAPTIVE) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_SHORT && p->mem_L < 1) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_ADAPTIVE && p->mem_a < 2) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_ADAPTIVE && p->adaptive_rule != FD_ADAPT_PAPER &&
        p->adaptive_rule != FD_ADAPT_PARTITION)
        return FD_ERR_INVALID_ARG;
    if (p->max_steps < 1 || p->max_steps > (1 << 28)) return FD_ERR_INVALID_ARG;
    if (p->ckpt_every < 0 || p->timeout_ms < 0) return FD_ERR_INVALID_ARG;
    if (p->tile_threads && (p->tile_threads < 32 || p->tile_threads > 512 || p->tile_threads % 32))
        return FD_ERR_INVALID_ARG;
    if (p->chunk_terms < 0 || p->stage_rows < 0 || p->stages < 0 || p->ctas_per_sm < 0)
        return FD_ERR_INVALID_ARG;
    if (p->stage_rows > 64 || p->stages > 16 || p->ctas_per_sm > 8) return FD_ERR_INVALID_ARG;
    if (p->head_lags < 0 || p->head_lags > 4096) return FD_ERR_INVALID_ARG;
    const bool kahan = p->flags & FD_FLAG_KAHAN;
    const bool adj = p->flags & FD_FLAG_KEEP_TAPE;
    if (!fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, kahan, false))
        return FD_ERR_UNSUPPORTED;
    if (adj && !fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, false, true)) return FD_ERR_UNSUPPORTED;
    if (closed_loop(*p)) {  // closed-loop adaptive memory: per-step kernel, history in state precision
        if (std::isnan(p->mem_tau) || p->mem_tau < 0.0) return FD_ERR_INVALID_ARG;
        if (p->mem_mode != FD_MEM_ADAPTIVE || p->hist_dtype != p->state_dtype || p->time_block || adj)
            return FD_ERR_UNSUPPORTED;
    }
    if (p->time_block) {
        const bool tc = tc_far(*p);
        if (p->time_block != 4 && p->time_block != 8 && p->time_block != 16 &&
            !(tc && (p->time_block == 32 || p->time_block == 64)))
            return (p->time_block == 32 || p->time_block == 64) ? FD_ERR_UNSUPPORTED : FD_ERR_INVALID_ARG;
        if (p->state_dtype != FD_F32 || p->accum_dtype != FD_F32 || kahan) return FD_ERR_UNSUPPORTED;
        if (!fdk::kernel_tb(p->time_block, adj, p->hist_dtype, tc)) return FD_ERR_UNSUPPORTED;
        if (tc) {  // point blocks of 128 (tile_threads 128 or 256), whole K slices of 16 rows per stage
            if (p->tile_threads && p->tile_threads != 128 && p->tile_threads != 256 && p->tile_threads != 512)
                return FD_ERR_INVALID_ARG;
            if (p->stage_rows && ((p->stage_rows != 16 && p->stage_rows != 32) || p->time_block % p->stage_rows))
                return FD_ERR_INVALID_ARG;
        }
        // arrival words hold a block generation (blocks / 4) and a chunk count in 16 bits each
        if ((int64_t)p->max_steps / p->time_block / 4 >= 65535) return FD_ERR_INVALID_ARG;
    }
    if (!(p->flags & FD_FLAG_ALLOW_UNSTABLE)) {
        // von Neumann bound of the full-memory scheme (checkerboard mode):
        // S * 4 ndim * sum_m psi_m (-1)^m = 2 with sum_m psi_m (-1)^m = 2^{1-g}
        const double S = p->alpha * std::pow(p->dt, p->gamma) / (p->dx * p->dx);
        if (S > std::pow(2.0, p->gamma) / (4.0 * p->ndim) * (1.0 + 1e-12)) return FD_ERR_UNSTABLE;
    }
    return FD_OK;
}

// ------------------------------------------------------------------- geometry

struct Geo {
    int threads, V, P, T, R, RS, NS, ctas, grid, maxC;
    int head;        // lags summed by the fixup
    int tb;          // temporal block (0: per-step kernel)
    int ub;          // blocked: one update unit per (block, tile)
    int cmax;        // blocked: most far chunks per block (0: chunks of R rows)
    int rwin;        // blocked: largest far chunk (rows), the coefficient window's length
    int nblocks;     // blocks of tb steps covering max_steps
    int tc;          // blocked: far units on the tensor cores
    int hplanes;     // history planes: 2 for FP32 history on the tensor cores (FP16 hi and lo), else 1
    int fsub;        // tensor cores: far units per (chunk, tile), each of P/fsub points (else 1)
    int nmtc;        // tensor cores, blocks of 32+: near and mid units on the tensor cores
    int lo_plane;    // the history stores a lo plane (paired FP32, or 16-bit history with nmtc)
    int halves;      // tensor cores: each CTA runs as two halves of `threads` threads
    size_t smem_half;  // tensor cores: dynamic shared memory of one half
    int tmem_cols;     // tensor cores: tensor-memory columns a CTA allocates (at most 512)
    int near;        // blocked, per-step update units, blocks of 16+: one near unit per (block, tile)
    int mid;         // blocked, near units, blocks of 32+: mid units per (block, tile), tb/16 - 1
    int ug;          // blocked: tiles per per-step update unit (tensor cores: 2)
    int ralign;      // blocked: far chunks start on multiples of ralign rows (tensor cores: RS)
    int hring_sep;   // separate state-precision head ring
    int hring_cap;
    int64_t hring_pitch;
    int sh, ss, sa;  // element sizes: history, state, accumulator
    int cap;
    int64_t pitch, part_pitch;
    size_t smem;
    int planes;
    int npar;        // partial-row parities
    // blocked, adaptive memory: first far row of each block (rows below it are tail rows of some
    // step of the block, whose weights change from step to step; the update units add them)
    std::vector<int> br0;
};

// Dynamic shared memory: stage ring, per-unit term tables (R coefficients x2, R slots), barriers,
// and for closed-loop memory the R + 1 entry offsets of a unit's terms and two doubles per warp.
inline size_t smem_bytes(const Geo &g, int rmax, bool closed = false)
{
    return (size_t)g.NS * g.RS * g.threads * 16 + (size_t)rmax * (2 * g.sa + 4) + 32 + 8 * (size_t)g.NS +
           (closed ? (size_t)(rmax + 1) * 4 + 8 + 16 * (size_t)(g.threads / 32) : 0);
}

// Blocked kernel: stage ring (block-long update units keep their steps' memory sums and their
// tile's state there, so it holds at least tb x planes + 2 rows, as the kernel assumes), four
// shifted copies of each coefficient window (psi, and psi' for the adjoint; with adaptive memory
// the first shifted copy holds the nonzero masks of the window's four-row groups), barriers.
inline size_t smem_bytes_tb(const Geo &g, int rwin, bool f16)
{
    const size_t ring = std::max((size_t)g.NS * g.RS * g.threads * 4 * g.sh, (size_t)(g.tb * g.planes + 2) * g.threads * 16);
    return ring + (size_t)g.planes * 4 * ((rwin + g.tb + 7) & ~3) * 4 + (f16 ? (size_t)rwin * 4 : 0) + 32 +
           8 * (size_t)g.NS;
}

// Tensor-core blocked kernel, one half of a CTA: stage ring (RS rows x P points of 16-bit history,
// in two planes for paired FP32 history), 1 KB-aligned; NS coefficient blocks (tb/8 1 KB atoms, hi and lo halves
// side by side); the coefficient window (and the row scales of FP16 or paired history; with paired
// history also the settled-weight window of a near or mid unit); 3 NS + 1
// barriers; rounded up to 1 KB.  The CTA takes two halves plus 1 KB of slack to align the base.
inline size_t smem_half_tc(const Geo &g, int rwin, bool scaled)
{
    const size_t ring = (size_t)g.NS * g.RS * (g.threads * 4 / g.fsub) * g.sh * g.hplanes;  // no block-long update units
    const size_t wr = (size_t)std::max(rwin, g.tb);  // a far chunk or a near unit's rows
    return align_up(align_up(ring, 1024) + (size_t)g.NS * (g.tb / 8) * 1024 +
                        (wr + g.tb + (scaled ? wr : 0) + (g.nmtc ? 2 * g.tb : 0)) * 4 + 16 +
                        8 * (size_t)(3 * g.NS + 1),
                    1024);
}

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// Last lag of step k whose weight is settled: adaptive memory gives lag m <= e(k) the weight
// g(m) of every later step (psi_m on the base interval, d psi_m at a median, 0 between medians,
// Definition 3.2); lags e(k)+1 .. k are the step's tail, weight psi_m (k <= a: e(k) = k).
inline int64_t settled_end(const int4 &e) { return std::max<int64_t>(e.x, (int64_t)e.z - 1); }

// Far rows [rlo, rhi) of block b of the blocked kernel: rows older than the previous block,
// limited to the short window; with adaptive memory, from the block's first settled row.
inline void block_rows(const fd_problem &p, const Geo &g, int64_t b, int64_t &rlo, int64_t &rhi)
{
    const int64_t kb = b * g.tb;
    rhi = std::max<int64_t>(0, kb - g.tb);
    rlo = (p.mem_mode == FD_MEM_SHORT)                                    ? std::max<int64_t>(0, kb - p.mem_L)
          : (p.mem_mode == FD_MEM_ADAPTIVE && b < (int64_t)g.br0.size()) ? g.br0[b]
                                                                         : 0;
    rlo = std::min(rlo, rhi);
}

// First row of a block's far chunks: its first far row, rounded down to a multiple of ralign on
// the tensor-core path (which streams whole stages; the rows below the far rows get weight 0).
inline int64_t block_origin(const Geo &g, int64_t lo) { return g.ralign > 1 ? lo - lo % g.ralign : lo; }

// Far chunking of block b: chunks of R rows, or, with cmax, of max(R, ceil(rows / cmax)) rows,
// so that a block-long update unit sums at most cmax partial rows per step.
inline void block_chunks(const fd_problem &p, const Geo &g, int64_t b, int64_t &Rb, int64_t &Cb)
{
    int64_t lo, hi;
    block_rows(p, g, b, lo, hi);
    const int64_t rows = hi - block_origin(g, lo);
    Rb = g.R;
    if (g.cmax) Rb = std::max<int64_t>(Rb, (rows + g.cmax - 1) / g.cmax);
    if (g.ralign > 1) Rb = (Rb + g.ralign - 1) / g.ralign * g.ralign;
    Cb = std::max<int64_t>(1, (rows + Rb - 1) / Rb);
}

void make_geo(const fd_problem &p, const Sched &s, int threads_override, Geo &g)
{
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
    g.tc = tc_far(p);
    // FP32 history on the tensor cores is stored as two FP16 planes (hi, lo) with row-tile scales
    g.hplanes = (g.tc && p.hist_dtype == FD_F32) ? 2 : 1;
    g.sh = g.hplanes == 2 ? 2 : dtype_size(p.hist_dtype);  // bytes of one stored element per plane
    g.ss = dtype_size(p.state_dtype);
    g.sa = dtype_size(p.accum_dtype);
    g.V = p.time_block ? 4 : 16 / g.sh;  // the blocked kernel keeps four points per thread
    g.planes = (p.flags & FD_FLAG_KEEP_TAPE) ? 2 : 1;
    int th = threads_override ? threads_override : p.tile_threads;
    if (!th) {
        th = 256;
        const int64_t need = (N + g.V - 1) / g.V;
        while (th > 64 && need <= th / 2) th /= 2;
    }
    // tensor cores: point blocks of 128, four warps per lane quarter, per half of a CTA
    if (g.tc) th = (th >= 256) ? 256 : 128;
    g.halves = g.tc ? 2 : 1;
    g.threads = th;
    g.P = th * g.V;
    g.T = (int)((N + g.P - 1) / g.P);
    // tensor cores: stages of 16 rows, or 32 for 16-bit history with blocks of 32+ (the bytes of a
    // near or mid unit's stage of 16 rows in two planes); as many as fit in 88 KB per half (2 .. 5)
    const int tc_rs = (g.tc && p.time_block % 32 == 0 && g.hplanes == 1) ? 32 : 16;
    g.RS = p.stage_rows ? p.stage_rows : g.tc ? tc_rs : 8;
    // near and mid units on the tensor cores: blocks of 32+, and a stage of 16 rows in two planes
    // the size of a far stage
    g.nmtc = g.tc && p.time_block >= 32 && g.RS * g.hplanes == 32;
    g.lo_plane = g.hplanes == 2 || g.nmtc;
    // Far sub-tiles: a tensor-core far unit covers P/fsub points, so that both halves' accumulators
    // (P/fsub/128 x tb columns each) fit the 512 tensor-memory columns and a stage of RS rows
    // (two planes for paired history) stays within 32 KB; the update units keep the whole tile.
    g.fsub = 1;
    if (g.tc)
        while (g.fsub < g.P / 128 &&
               ((g.P / g.fsub / 128) * p.time_block > 256 || (size_t)g.RS * (g.P / g.fsub) * 2 * g.hplanes > (32u << 10)))
            g.fsub *= 2;
    // (a tensor-core stage: RS rows of history plus its coefficient block)
    g.NS = p.stages ? p.stages
           : g.tc   ? std::max(2, std::min(5, (88 << 10) / (g.RS * (g.P / g.fsub) * g.sh * g.hplanes + (p.time_block / 8) * 1024)))
                    : 3;
    g.ctas = p.ctas_per_sm ? p.ctas_per_sm : 2;
    g.ralign = g.tc ? g.RS : 1;
    int sms = device_sms();
    if (sms <= 0) sms = 152;
    g.grid = sms * g.ctas * g.halves;  // units are processed by grid (half-)CTAs
    g.cap = p.max_steps;
    // short memory keeps a ring of L+1 rows, unless the adjoint's recompute will read old rows
    // (the tensor-map copies of the tensor-core path take whole stages, so they keep every row)
    if (p.mem_mode == FD_MEM_SHORT && !(p.flags & FD_FLAG_KEEP_TAPE) && !g.tc)
        g.cap = (int)std::min<int64_t>((int64_t)p.mem_L + 1, p.max_steps);
    g.cap = std::max(g.cap, 1);
    g.hring_sep = (p.hist_dtype != p.state_dtype) || g.hplanes == 2;
    g.head = p.head_lags ? p.head_lags : (g.hring_sep ? 32 : 8);
    if (!g.hring_sep && g.cap < g.head + 1) g.head = std::max(1, g.cap - 1);
    int64_t nmax = 0;
    for (const int4 &e : s.step) nmax = std::max(nmax, n_terms(e) - std::min<int64_t>(g.head, e.x));
    if (adaptive_adjoint(p) && p.max_steps > 1)  // the adjoint's steps have full memory's terms
        nmax = std::max(nmax, (int64_t)(p.max_steps - 1) - std::min<int64_t>(g.head, p.max_steps - 1));
    if (p.chunk_terms) {
        g.R = p.chunk_terms;
    } else {
        int64_t r = (nmax * g.T + 4LL * g.grid - 1) / (4LL * g.grid);
        r = std::max<int64_t>(r, 2 * g.RS);
        r = std::min<int64_t>(r, 256);
        r = (r + g.RS - 1) / g.RS * g.RS;
        g.R = (int)r;
    }
    g.maxC = (int)std::max<int64_t>(1, (nmax + g.R - 1) / g.R);
    g.tb = p.time_block;
    g.npar = npar_for(g.tb);
    g.nblocks = g.tb ? (p.max_steps + g.tb - 1) / g.tb : 0;
    g.ub = 0;
    g.near = 0;
    g.mid = 0;
    g.ug = 1;
    g.smem_half = 0;
    g.cmax = 0;
    g.rwin = g.R;
    g.br0.clear();
    if (g.tb) {
        if (p.mem_mode == FD_MEM_ADAPTIVE) {
            // rows 0 .. k-e(k)-1 are step k's tail: far rows start above every step's tail
            g.br0.assign(g.nblocks, 0);
            for (int64_t b = 0; b < g.nblocks; ++b)
                for (int64_t k = b * g.tb; k < std::min<int64_t>((b + 1) * g.tb, p.max_steps); ++k)
                    g.br0[b] = (int)std::max<int64_t>(g.br0[b], k - settled_end(s.step[k]));
        }
        // (with the adjoint of adaptive memory, also the full-memory blocks the adjoint runs)
        const fd_problem pf = full_memory(p);
        const int nprob = adaptive_adjoint(p) ? 2 : 1;
        int64_t rmax = 0;
        for (int ip = 0; ip < nprob; ++ip)
            for (int64_t b = 0; b < g.nblocks; ++b) {
                int64_t lo, hi;
                block_rows(ip ? pf : p, g, b, lo, hi);
                rmax = std::max(rmax, hi - lo);
            }
        if (!p.chunk_terms) {
            int64_t r = (rmax * g.T + 4LL * g.grid - 1) / (4LL * g.grid);
            r = std::min<int64_t>(std::max<int64_t>(r, 2 * g.RS), 512);
            if (g.tc) {
                // tensor cores: long chunks, as each chunk writes tb FP32 partial rows and every
                // update reads one per chunk: about two far units per half-CTA and block, up to
                // the longest chunk whose coefficient window two halves still hold in shared
                // memory (config 3: 3072-row chunks 3% faster than 2048)
                int64_t cap = 4096;
                while (cap > 1024 && 2 * smem_half_tc(g, (int)cap, p.hist_dtype != FD_BF16) + 1024 > (223u << 10))
                    cap -= 512;
                r = (rmax * g.T * g.fsub + 2LL * sms * g.halves - 1) / (2LL * sms * g.halves);
                r = std::min<int64_t>(std::max<int64_t>(r, 2 * g.RS), cap);
            }
            g.R = (int)((r + g.RS - 1) / g.RS * g.RS);
        }
        if (g.ralign > 1) g.R = (g.R + g.ralign - 1) / g.ralign * g.ralign;
        // Block-long update units need every tile's unit resident at once: allow them when the
        // tiles are at most a quarter of the SMs, so at least three quarters keep streaming.
        // (the tensor-core kernels have none)
        g.ub = !(p.flags & FD_FLAG_STEP_UPDATES) && !g.tc && (int64_t)g.T * 4 <= sms;
        g.cmax = g.ub ? std::max(1, 128 / g.tb) : 0;
        int64_t cmaxb = 1, rwin = g.R;
        for (int ip = 0; ip < nprob; ++ip)
            for (int64_t b = 0; b < g.nblocks; ++b) {
                int64_t Rb, Cb;
                block_chunks(ip ? pf : p, g, b, Rb, Cb);
                cmaxb = std::max(cmaxb, Cb);
                rwin = std::max(rwin, Rb);
            }
        // Near units: with per-step update units and blocks of 16 or more, the previous block's
        // rows enter each step through one partial row (after the far chunks') instead of as
        // TB head lags read by every step's update
        g.near = !g.ub && g.tb >= 16;
        // Mid units: with blocks of 32 or more, sub-block j = 1 .. tb/16-1 (16 steps each) gets the
        // block's rows before it as one more partial row, so an update sums at most 15 head lags
        g.mid = (g.near && g.tb >= 32) ? g.tb / 16 - 1 : 0;
        // Tensor-core kernels with more tiles than half the grid's half-CTAs: two tiles per
        // per-step update unit, so that a step's update units (T/2) leave half-CTAs free to claim
        // the next step's while this one finishes (with fewer tiles the second tile's phase B
        // would only lengthen the step-to-step chain)
        g.ug = (g.tc && !g.ub && (int64_t)g.T * 2 > (int64_t)sms * g.halves) ? 2 : 1;  // (one CTA per SM)
        g.maxC = (int)cmaxb + g.near + (g.mid ? 1 : 0);
        g.rwin = (int)rwin;
    }
    g.pitch = (int64_t)align_up((size_t)N * g.sh, kAlign);
    // low-precision history keeps its newest rows in FP32 too: the per-step kernel its head lags,
    // the blocked kernel the rows of the current and the previous block
    g.hring_cap = !g.hring_sep ? g.cap : g.tb ? 2 * g.tb : g.head + 1;
    g.hring_pitch = g.hring_sep ? (int64_t)align_up(align_up((size_t)N, 8) * g.ss, kAlign) : g.pitch;
    g.part_pitch = (int64_t)align_up((size_t)(align_up((size_t)N, 8)) * g.sa, kAlign);
    g.tmem_cols = 0;
    if (g.tc) {  // each half allocates P/fsub/128 x tb tensor-memory columns (a power of two) of 512
        int cols = 32;
        while (cols < (g.P / g.fsub / 128) * g.tb) cols *= 2;
        g.tmem_cols = cols * g.halves;
        g.ctas = std::max(1, std::min(g.ctas, 512 / (cols * g.halves)));
        g.smem_half = smem_half_tc(g, g.rwin, p.hist_dtype != FD_BF16);
    }
    g.smem = g.tc ? g.halves * g.smem_half + 1024 : g.tb ? smem_bytes_tb(g, g.rwin, p.hist_dtype == FD_F16) : smem_bytes(g, g.R, closed_loop(p));
}

// Units per step: T tiles x max(1, ceil(n(k)/R)) chunks.
inline int64_t step_units(const Geo &g, const int4 &e)
{
    const int64_t n = n_terms(e) - std::min<int64_t>(g.head, e.x);
    return (int64_t)g.T * std::max<int64_t>(1, (n + g.R - 1) / g.R);
}

// Near and mid units per (block, tile): on the tensor cores, one per far sub-tile.
inline int nsub_of(const Geo &g) { return g.nmtc ? g.fsub : 1; }

// Units of group b of the blocked kernel: the far chunks of block b (none past the last block)
// plus block b-1's update units (one per step and tile, or one per tile for the whole block).
inline int64_t block_units(const fd_problem &p, const Geo &g, int64_t b)
{
    int64_t far = 0;
    if (b < g.nblocks) {
        int64_t Rb, Cb;
        block_chunks(p, g, b, Rb, Cb);
        far = (int64_t)g.T * (Cb * g.fsub + g.near * nsub_of(g));  // far chunks (fsub units each), near units
    }
    const int64_t tg = (g.T + g.ug - 1) / g.ug;  // update units per step
    return far + (b >= 1 ? (g.ub ? (int64_t)g.T : tg * g.tb) + (int64_t)g.T * g.mid * nsub_of(g) : 0);
}

// History rows the blocked kernel reads over max_steps steps: the far rows once per block, then
// every step's head rows (lags 1 .. min(k - kb + tb, n(k)); with near units the block's own rows,
// with mid units those of its own sub-block of 16 steps, plus the near and mid units' rows once
// each), or, with block-long update units, the previous block's rows once per block.
int64_t blocked_stream_rows(const fd_problem &p, const Geo &g, int64_t *head_rows = nullptr)
{
    const int tb = g.tb;
    int64_t st = 0, hd = 0;
    for (int64_t b = 0; b < g.nblocks; ++b) {
        int64_t lo, hi;
        block_rows(p, g, b, lo, hi);
        st += hi - block_origin(g, lo);
        // block-long update units read the previous block's rows once; later rows stay on chip
        if (g.ub) hd += std::min<int64_t>(tb, b * tb);
        // adaptive tail rows below the far rows: once per block-long unit, else once per step
        if (p.mem_mode == FD_MEM_ADAPTIVE)
            st += (int64_t)std::min<int64_t>(lo, (int64_t)g.br0[b]) *
                  (g.ub ? 1 : std::min<int64_t>(tb, p.max_steps - b * tb));
    }
    if (!g.ub)
        for (int64_t k = 0; k < p.max_steps; ++k) {
            const int64_t nb = (p.mem_mode == FD_MEM_SHORT) ? std::min<int64_t>(p.mem_L, k) : k;
            const int64_t t = k - (k / tb) * tb;
            hd += std::min<int64_t>(g.near ? (g.mid ? t % 16 : t) : t + tb, nb);
            if (g.near && t == 0) hd += std::min<int64_t>(tb, k);  // the near unit's rows, once per block
            if (g.mid && t > 0 && t % 16 == 0) hd += t;             // a mid unit's rows, once per sub-block
        }
    if (head_rows) *head_rows = hd;
    return st + hd;
}

// Adjoint of adaptive memory: every step's tail terms (lags m beyond its settled end e(k), weight
// psi_m where the adjoint uses g(m)), grouped by the adjoint row r = k - m they reach, ascending in k
// within a row (Definitions 3.1/3.2, Proposition 3.1).  With weights, each entry carries
// psi_m - g(m) and the same for the gamma derivatives; without, only the layout is computed.
struct TailList {
    std::vector<int> off;  // rows + 1 offsets
    std::vector<fdk::AdjTail> e;
};
void tail_terms(const Sched &s, const std::vector<double> *psi, const std::vector<double> *dpsi,
                const std::vector<double> *gw, const std::vector<double> *dgw, TailList &t)
{
    const int64_t K = (int64_t)s.step.size();
    int64_t rows = 0;
    for (int64_t k = 0; k < K; ++k) rows = std::max(rows, k - settled_end(s.step[k]));
    t.off.assign((size_t)rows + 1, 0);
    for (int64_t k = 0; k < K; ++k)
        for (int64_t r = 0; r < k - settled_end(s.step[k]); ++r) ++t.off[(size_t)r + 1];
    for (int64_t r = 0; r < rows; ++r) t.off[(size_t)r + 1] += t.off[(size_t)r];
    t.e.assign((size_t)t.off[(size_t)rows], fdk::AdjTail{0, 0, 0.0, 0.0});
    std::vector<int> cur(t.off.begin(), t.off.end() - 1);
    for (int64_t k = 0; k < K; ++k)
        for (int64_t r = 0; r < k - settled_end(s.step[k]); ++r) {
            fdk::AdjTail &x = t.e[(size_t)cur[(size_t)r]++];
            const int64_t m = k - r;
            x.k = (int)k;
            if (psi) {
                x.w = (*psi)[m] - (*gw)[m];
                x.w2 = (*dpsi)[m] - (*dgw)[m];
            }
        }
}

// Device-side layout of one instance inside the workspace.
struct Layout {
    char *ubuf[2];
    char *ulo[2], *alo[2], *rlo[2];  // compensated-state low parts (forward, adjoint, recompute)
    char *hist;
    char *hring;
    float *hscale;
    char *part;
    unsigned *arrive, *done;
    char *psi, *dpsi, *gcoef;
    char *gw;  // blocked, adaptive memory: settled weight g(m) of every lag
    int *glag, *br0;
    int4 *sched;
    char *tmap;  // tensor-core path: tensor map of the history rows (128 bytes, 64-byte aligned)
    char *tmap2;  // tensor-core near / mid units over 16-bit history: both planes, 16-row boxes
    // adjoint of adaptive memory: d/dgamma of the settled weights, the full-memory schedule the
    // per-step adjoint runs, and the tail terms by adjoint row
    char *dgw;
    int4 *asched;
    int *acorr_off;
    fdk::AdjTail *acorr;
    int acorr_rows;
    // adjoint
    char *ckpt, *seg, *rec[2], *ahist, *abuf[2];
    double *dots;
    int ckpt_rows, seg_rows;
    // closed-loop adaptive memory: row maxima D, M and the tiles counted into them (max_steps rows
    // each), the terms counter, the increment length of each median
    double *clD, *clM;
    unsigned *clrows;
    unsigned long long *clterms;
    int *gd;
    // the ring of per-step decisions: a + 1 slots of per-median lengths and per-chunk words
    unsigned char *clcnt;
    unsigned long long *clword;
    int clslots, clgmax;
};

void carve_instance(Carve &c, const fd_problem &p, const Geo &g, const Sched &s, Layout &L,
                    unsigned *counters = nullptr, bool external_counters = false)
{
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
    const size_t ubytes = align_up((size_t)N * g.ss, kAlign);
    L.ubuf[0] = c.take(ubytes);
    L.ubuf[1] = c.take(ubytes);
    const bool comp = p.state_dtype == FD_F32 && !(p.flags & FD_FLAG_PLAIN_STATE);
    const bool adj = p.flags & FD_FLAG_KEEP_TAPE;
    for (int i = 0; i < 2; ++i) {
        L.ulo[i] = comp ? c.take(ubytes) : nullptr;
        L.alo[i] = (comp && adj) ? c.take(ubytes) : nullptr;
        L.rlo[i] = (comp && adj) ? c.take(ubytes) : nullptr;
    }
    L.hist = c.take((size_t)g.cap * g.pitch * (g.lo_plane ? 2 : 1));
    L.hring = g.hring_sep ? c.take((size_t)g.hring_cap * g.hring_pitch) : L.hist;
    // power-of-two scales per (row, tile): FP16 history, and paired FP32 history
    L.hscale = (p.hist_dtype == FD_F16 || g.hplanes == 2)
                   ? (float *)c.take((size_t)g.cap * g.T * sizeof(float))
                   : nullptr;
    L.part = c.take((size_t)g.npar * g.maxC * g.planes * std::max(1, g.tb) * g.part_pitch);
    L.arrive = external_counters ? counters
                                 : (unsigned *)c.take(sizeof(unsigned) * (g.npar + 1) * (size_t)g.T);
    L.done = L.arrive ? L.arrive + g.npar * g.T : nullptr;
    L.psi = c.take((size_t)(p.max_steps + 1 + 2 * g.tb) * g.sa);  // blocked: windows read lags up to 2 tb (near units)
    L.dpsi = (p.flags & FD_FLAG_KEEP_TAPE) ? c.take((size_t)(p.max_steps + 1 + 2 * g.tb) * g.sa) : nullptr;
    L.sched = (int4 *)c.take(sizeof(int4) * (size_t)p.max_steps);
    const size_t ng = std::max<size_t>(1, s.G.size());
    L.glag = (int *)c.take(sizeof(int) * ng);
    L.gcoef = c.take((size_t)g.sa * ng);
    const bool btab = g.tb && p.mem_mode == FD_MEM_ADAPTIVE, aad = adaptive_adjoint(p);
    const size_t wlen = (size_t)(p.max_steps + 1 + 2 * g.tb) * g.sa;
    L.gw = (btab || aad) ? c.take(wlen) : nullptr;
    L.br0 = btab ? (int *)c.take(sizeof(int) * (size_t)(g.nblocks + 1)) : nullptr;
    L.dgw = aad ? c.take(wlen) : nullptr;
    L.asched = (aad && !g.tb) ? (int4 *)c.take(sizeof(int4) * (size_t)p.max_steps) : nullptr;
    L.acorr_off = nullptr;
    L.acorr = nullptr;
    L.acorr_rows = 0;
    if (aad) {
        TailList tl;
        tail_terms(s, nullptr, nullptr, nullptr, nullptr, tl);
        L.acorr_rows = (int)tl.off.size() - 1;
        L.acorr_off = (int *)c.take(sizeof(int) * tl.off.size());
        L.acorr = (fdk::AdjTail *)c.take(sizeof(fdk::AdjTail) * std::max<size_t>(1, tl.e.size()));
    }
    L.tmap = g.tc ? c.take(128) : nullptr;
    L.tmap2 = (g.nmtc && g.hplanes == 1) ? c.take(128) : nullptr;
    L.clD = L.clM = nullptr;
    L.clrows = nullptr;
    L.clterms = nullptr;
    L.gd = nullptr;
    L.clcnt = nullptr;
    L.clword = nullptr;
    L.clslots = L.clgmax = 0;
    if (closed_loop(p)) {
        L.clD = (double *)c.take(sizeof(double) * (size_t)p.max_steps);
        L.clM = (double *)c.take(sizeof(double) * (size_t)p.max_steps);
        L.clrows = (unsigned *)c.take(sizeof(unsigned) * (size_t)p.max_steps);
        L.clterms = (unsigned long long *)c.take(sizeof(unsigned long long));
        L.gd = (int *)c.take(sizeof(int) * ng);
        L.clslots = p.mem_a + 1;
        L.clgmax = (int)ng;
        L.clcnt = (unsigned char *)c.take((size_t)L.clslots * ng);
        L.clword = (unsigned long long *)c.take(sizeof(unsigned long long) * (size_t)L.clslots * g.maxC);
    }
    L.ckpt = L.seg = L.rec[0] = L.rec[1] = L.ahist = L.abuf[0] = L.abuf[1] = nullptr;
    L.dots = nullptr;
    L.ckpt_rows = L.seg_rows = 0;
    if (p.flags & FD_FLAG_KEEP_TAPE) {
        const int C = p.ckpt_every ? p.ckpt_every : 200;
        L.ckpt_rows = p.max_steps / C + 1;
        L.seg_rows = std::min(C, p.max_steps);
        L.ckpt = c.take((size_t)L.ckpt_rows * N * g.ss);
        L.seg = c.take((size_t)L.seg_rows * N * g.ss);
        L.rec[0] = c.take(ubytes);
        L.rec[1] = c.take(ubytes);
        L.ahist = c.take((size_t)p.max_steps * g.pitch);
        L.abuf[0] = c.take(ubytes);
        L.abuf[1] = c.take(ubytes);
        L.dots = (double *)c.take(sizeof(double) * 8 * (size_t)g.T);
    }
}

// Control words shared by every launch of a handle / batch.
struct Ctrl {
    unsigned long long *queue;
    int *err;
    unsigned *nonfinite;
    long long *err_info;  // 8 words: the first wait that gave up (site, operands, CTA)
};

Ctrl carve_ctrl(Carve &c)
{
    char *b = c.take(256);
    Ctrl r;
    r.queue = (unsigned long long *)b;
    r.err = b ? (int *)(b + 64) : nullptr;
    r.nonfinite = b ? (unsigned *)(b + 128) : nullptr;
    r.err_info = b ? (long long *)(b + 192) : nullptr;
    return r;
}

// Host-side tables of an instance, converted to the accumulator type.
struct Tables {
    std::vector<double> psi, dpsi;
    std::vector<unsigned char> psi_a, dpsi_a, gcoef_a, gw_a, dgw_a;
    std::vector<int> glag, br0, gd;
    std::vector<int4> asched;
    TailList tail;
};

template <class TA> void to_acc(const std::vector<double> &x, std::vector<unsigned char> &out)
{
    out.resize(x.size() * sizeof(TA));
    TA *o = reinterpret_cast<TA *>(out.data());
    for (size_t i = 0; i < x.size(); ++i) o[i] = (TA)x[i];
}

void build_tables(const fd_problem &p, const Sched &s, const Geo &g, Tables &t)
{
    const int64_t n = (int64_t)p.max_steps + 1 + 2 * g.tb;
    t.psi.resize(n);
    t.dpsi.resize(n);
    gl_weights(p.gamma, n, t.psi.data(), t.dpsi.data());
    std::vector<double> gc(std::max<size_t>(1, s.G.size()), 0.0);
    t.glag.assign(gc.size(), 0);
    t.gd.assign(gc.size(), 1);
    for (size_t i = 0; i < s.G.size(); ++i) {
        gc[i] = (double)s.G[i].mult * t.psi[s.G[i].lag];
        t.glag[i] = s.G[i].lag;
        t.gd[i] = s.G[i].mult;
    }
    // blocked adaptive memory: g(m) = psi_m on the base interval [0, a], d psi_m at a median,
    // 0 at the other lags (each median's weight, as the per-step schedule uses it)
    // adjoint of adaptive memory: dg/dgamma likewise (d psi'_m at a median), the full-memory
    // schedule of the per-step adjoint, and the tail terms
    std::vector<double> gw, dgw;
    if ((g.tb && p.mem_mode == FD_MEM_ADAPTIVE) || adaptive_adjoint(p)) {
        gw.assign(n, 0.0);
        dgw.assign(n, 0.0);
        for (int64_t m = 0; m <= std::min<int64_t>(p.mem_a, n - 1); ++m) {
            gw[m] = t.psi[m];
            dgw[m] = t.dpsi[m];
        }
        for (size_t i = 0; i < s.G.size(); ++i)
            if (s.G[i].lag < n) {
                gw[s.G[i].lag] = gc[i];
                dgw[s.G[i].lag] = (double)s.G[i].mult * t.dpsi[s.G[i].lag];
            }
        if (g.tb) {
            t.br0 = g.br0;
            t.br0.push_back(0);
        }
    }
    if (adaptive_adjoint(p)) {
        if (!g.tb)
            for (int64_t k = 0; k < p.max_steps; ++k) t.asched.push_back(full_step(k));
        tail_terms(s, &t.psi, &t.dpsi, &gw, &dgw, t.tail);
    }
    if (g.sa == 8) {
        to_acc<double>(t.psi, t.psi_a);
        to_acc<double>(t.dpsi, t.dpsi_a);
        to_acc<double>(gc, t.gcoef_a);
        to_acc<double>(gw, t.gw_a);
        to_acc<double>(dgw, t.dgw_a);
    } else {
        to_acc<float>(t.psi, t.psi_a);
        to_acc<float>(t.dpsi, t.dpsi_a);
        to_acc<float>(gc, t.gcoef_a);
        to_acc<float>(gw, t.gw_a);
        to_acc<float>(dgw, t.dgw_a);
    }
}

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            (void)cudaGetLastError();              \
            return FD_ERR_CUDA;                    \
        }                                          \
    } while (0)

int upload_tables(const fd_problem &p, const Sched &s, const Tables &t, const Layout &L, cudaStream_t st)
{
    CK(cudaMemcpyAsync(L.psi, t.psi_a.data(), t.psi_a.size(), cudaMemcpyHostToDevice, st));
    if (L.dpsi) CK(cudaMemcpyAsync(L.dpsi, t.dpsi_a.data(), t.dpsi_a.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.sched, s.step.data(), sizeof(int4) * s.step.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.glag, t.glag.data(), sizeof(int) * t.glag.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.gcoef, t.gcoef_a.data(), t.gcoef_a.size(), cudaMemcpyHostToDevice, st));
    if (L.gd) CK(cudaMemcpyAsync(L.gd, t.gd.data(), sizeof(int) * t.gd.size(), cudaMemcpyHostToDevice, st));
    if (L.gw) CK(cudaMemcpyAsync(L.gw, t.gw_a.data(), t.gw_a.size(), cudaMemcpyHostToDevice, st));
    if (L.br0) CK(cudaMemcpyAsync(L.br0, t.br0.data(), sizeof(int) * t.br0.size(), cudaMemcpyHostToDevice, st));
    if (L.dgw) CK(cudaMemcpyAsync(L.dgw, t.dgw_a.data(), t.dgw_a.size(), cudaMemcpyHostToDevice, st));
    if (L.asched)
        CK(cudaMemcpyAsync(L.asched, t.asched.data(), sizeof(int4) * t.asched.size(), cudaMemcpyHostToDevice, st));
    if (L.acorr_off) {
        CK(cudaMemcpyAsync(L.acorr_off, t.tail.off.data(), sizeof(int) * t.tail.off.size(), cudaMemcpyHostToDevice, st));
        if (!t.tail.e.empty())
            CK(cudaMemcpyAsync(L.acorr, t.tail.e.data(), sizeof(fdk::AdjTail) * t.tail.e.size(), cudaMemcpyHostToDevice,
                               st));
    }
    (void)p;
    return FD_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor-core path: the history rows as a 16-bit tensor (BF16, FP16, or the hi and lo FP16 planes
// of paired FP32 history as one tensor of 2 cap rows) read with the 128-byte swizzle the MMA's A
// operand expects, in boxes of 64 points (128 bytes) x RS rows.  Preferred: a 3-D view (64 points,
// rows, groups of 64 points; the group stride of 128 bytes is below the row pitch) whose one box
// per stage covers all P/64 groups of a tile.  If the driver refuses that view, a 2-D view
// (points, rows) with one box per group.  Points past the padded row read as zeros.  Encoded on
// the host, copied into the workspace; returns the rank used (0 on failure).  `planes` planes of
// cap rows each (the lo plane follows the rows), boxes of `box_rows` rows.
int encode_tmap(const Geo &g, const Layout &L, CUtensorMap *m, int hist, int planes, int box_rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return 0;
    // (paired FP32 history: FP16, both planes as one tensor of 2 cap rows)
    const CUtensorMapDataType dt =
        hist == FD_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t rows = (cuuint64_t)g.cap * planes;
    {
        const cuuint64_t dims[3] = {64u, rows, (cuuint64_t)(g.pitch / 128)};
        const cuuint64_t strides[2] = {(cuuint64_t)g.pitch, 128u};
        const cuuint32_t box[3] = {64u, (cuuint32_t)box_rows, (cuuint32_t)(g.P / g.fsub / 64)};
        const cuuint32_t es[3] = {1u, 1u, 1u};
        if (enc(m, dt, 3, L.hist, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
            CUDA_SUCCESS)
            return 3;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)(g.pitch / 2), rows};
    const cuuint64_t strides[1] = {(cuuint64_t)g.pitch};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1u, 1u};
    if (enc(m, dt, 2, L.hist, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
        CUDA_SUCCESS)
        return 2;
    return 0;
}

int upload_tmap(const fd_problem &p, const Geo &g, const Layout &L, Inst &I, cudaStream_t st)
{
    if (!g.tc) return FD_OK;
    alignas(64) CUtensorMap m, m2;
    I.tmap_rank = encode_tmap(g, L, &m, p.hist_dtype, g.hplanes, g.RS);
    if (!I.tmap_rank) return FD_ERR_CUDA;
    CK(cudaMemcpyAsync(L.tmap, &m, sizeof(m), cudaMemcpyHostToDevice, st));
    if (L.tmap2) {  // near and mid units over 16-bit history: both planes in boxes of 16 rows
        I.tmap2_rank = encode_tmap(g, L, &m2, p.hist_dtype, 2, 16);
        if (!I.tmap2_rank) return FD_ERR_CUDA;
        CK(cudaMemcpyAsync(L.tmap2, &m2, sizeof(m2), cudaMemcpyHostToDevice, st));
    }
    return FD_OK;
}

Inst make_inst(const fd_problem &p, const Geo &g, const Layout &L, bool adj)
{
    Inst I;
    std::memset(&I, 0, sizeof(I));
    I.ndim = p.ndim;
    I.nx = p.nx;
    I.ny = p.ny;
    I.bc = p.bc;
    I.N = p.nx * p.ny * p.nz;
    I.nz = p.nz;
    I.T = g.T;
    I.P = g.P;
    I.R = g.R;
    I.hist_write = 1;
    I.cap = adj ? p.max_steps : g.cap;
    I.maxC = g.maxC;
    I.tb = g.tb;
    I.mem_mode = p.mem_mode;
    I.mem_L = p.mem_L;
    I.ksteps = p.max_steps;
    I.ub = g.ub;
    I.cmax = g.cmax;
    I.ralign = g.ralign;
    I.near = g.near;
    I.ug = g.ug;
    I.mid = g.mid;
    I.tmap = L.tmap;
    I.tmap2 = L.tmap2;
    I.lo_plane = g.lo_plane && !adj;
    if (g.tc) {  // tensor-memory columns per half: the geometry's (at most 256, checked at init)
        I.tc_cols = g.tmem_cols / g.halves;
    }
    I.npar = g.npar;
    I.stall = (p.flags & FD_FLAG_INJECT_STALL) ? 1 : 0;
    I.tape_every = 1;
    I.S = p.alpha * std::pow(p.dt, p.gamma) / (p.dx * p.dx);
    I.dt = p.dt;
    for (int i = 0; i < 4; ++i) I.react[i] = p.react[i];
    I.pitch = g.pitch;
    I.part_pitch = g.part_pitch;
    I.hist = adj ? L.ahist : L.hist;
    I.head = g.head;
    I.hring_sep = adj ? 0 : g.hring_sep;
    I.hring = adj ? L.ahist : L.hring;
    I.hring_cap = adj ? p.max_steps : g.hring_cap;
    I.hring_pitch = adj ? g.pitch : g.hring_pitch;
    I.hscale = adj ? nullptr : L.hscale;
    I.ubuf[0] = adj ? L.abuf[0] : L.ubuf[0];
    I.ubuf[1] = adj ? L.abuf[1] : L.ubuf[1];
    I.ulo[0] = adj ? L.alo[0] : L.ulo[0];
    I.ulo[1] = adj ? L.alo[1] : L.ulo[1];
    I.part = L.part;
    I.arrive = L.arrive;
    I.done = L.done;
    I.psi = L.psi;
    I.dpsi = L.dpsi;
    I.sched = L.sched;
    I.g_lag = L.glag;
    I.g_coef = L.gcoef;
    I.gw = L.gw;
    I.br0 = L.br0;
    if (!adj && L.clD) {
        I.cl_D = L.clD;
        I.cl_M = L.clM;
        I.cl_rows = L.clrows;
        I.cl_terms = L.clterms;
        I.g_d = L.gd;
        I.cl_tau = p.mem_tau;
        // every increment lies above the base interval [0, a] (both rules): none reaches a lag
        // below a + 1
        I.cl_lo = p.mem_a + 1;
        I.cl_cnt = L.clcnt;
        I.cl_word = L.clword;
        I.cl_slots = L.clslots;
        I.cl_gmax = L.clgmax;
    }
    if (!adj && L.ckpt) {
        I.tape = L.ckpt;
        I.tape_k0 = 0;
        I.tape_every = p.ckpt_every ? p.ckpt_every : 200;
        I.tape_rows = L.ckpt_rows;
    }
    if (adj) {
        I.stall = 0;
        I.uadj = L.seg;
        I.dots = L.dots;
    }
    if (adj && p.mem_mode == FD_MEM_ADAPTIVE) {
        // full memory with the settled weights g(m), dg/dgamma, plus the tail terms
        I.psi = L.gw;
        I.dpsi = L.dgw;
        I.mem_mode = FD_MEM_FULL;
        I.gw = nullptr;
        I.br0 = nullptr;
        if (L.asched) I.sched = L.asched;
        I.acorr_off = L.acorr_off;
        I.acorr = L.acorr;
        I.acorr_rows = L.acorr_rows;
    }
    return I;
}

// The attribute is per kernel and process-wide, while handles with different geometries share a
// kernel: allow the device's opt-in maximum once, then check each handle's need against it.
int set_smem_attr(const void *fn, size_t smem)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    if (smem + 4096 > (size_t)optin) return FD_ERR_INVALID_ARG;  // static shared memory needs room too
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 4096) != cudaSuccess) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    return FD_OK;
}

int resolve_grid(const void *fn, Geo &g)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, g.threads * g.halves, g.smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    if (occ < 1) return FD_ERR_INVALID_ARG;  // stage ring does not fit in shared memory
    g.ctas = std::min(g.ctas, occ);
    int sms = device_sms();
    if (sms <= 0) return FD_ERR_CUDA;
    g.grid = sms * g.ctas * g.halves;
    return FD_OK;
}

int status_from(int err, unsigned nonfinite)
{
    if (err == fdk::ERR_TIMEOUT || err == fdk::ERR_PIPE) return FD_ERR_TIMEOUT;
    if (nonfinite) return FD_ERR_NONFINITE;
    return FD_OK;
}

}  // namespace

// ================================================================== handle

struct fd_handle {
    fd_problem p;
    cudaStream_t st;
    char *ws;
    size_t ws_bytes;
    Geo g;
    Sched s;
    Tables t;
    Layout L;
    Ctrl ctrl;
    char *ctrl_zero_base;    // counters region to clear per launch
    size_t ctrl_zero_bytes;
    Inst inst_fwd, inst_adj;
    Inst *d_inst;            // [0] forward, [1] adjoint / recompute scratch
    long long *d_goff;
    int2 *d_ginfo;
    std::vector<long long> goff;
    // adjoint of adaptive memory: the adjoint's groups (full memory's units)
    long long *d_agoff;
    int2 *d_aginfo;
    std::vector<long long> agoff;
    const void *kfwd, *kadj;
    int64_t k;
    int bad;                 // state invalid after a failed launch
};

static int launch(fd_handle *h, const void *fn, const Inst *d_inst, int g_begin, int g_end, int k0,
                  int k_end = 0, bool adj_groups = false)
{
    const bool ag = adj_groups && h->d_agoff;
    const std::vector<long long> &goff = ag ? h->agoff : h->goff;
    Launch L;
    std::memset(&L, 0, sizeof(L));
    L.inst = d_inst;
    L.g_off = ag ? h->d_agoff : h->d_goff;
    L.g_info = ag ? h->d_aginfo : h->d_ginfo;
    L.g_begin = g_begin;
    L.g_end = g_end;
    L.k0 = k0;
    L.k_end = k_end;
    L.stage_rows = h->g.RS;
    L.stages = h->g.NS;
    L.rmax = h->g.tb ? h->g.rwin : h->g.R;
    L.smem_half = (int)h->g.smem_half;
    L.fsub = h->g.fsub;
    L.nm_tc = h->g.nmtc;
    L.queue = h->ctrl.queue;
    L.err = h->ctrl.err;
    L.nonfinite = h->ctrl.nonfinite;
    L.err_info = h->ctrl.err_info;
    L.timeout_ns = (long long)(h->p.timeout_ms ? h->p.timeout_ms : 10000) * 1000000LL;
    CK(cudaMemsetAsync(h->ctrl.queue, 0, sizeof(unsigned long long), h->st));
    CK(cudaMemsetAsync(h->ctrl_zero_base, 0, h->ctrl_zero_bytes, h->st));
    const int64_t units = goff[g_end] - goff[g_begin];
    const int hv = h->g.halves;
    const int grid = (int)((std::min<int64_t>(h->g.grid, units) + hv - 1) / hv);
    void *args[] = {&L};
    CK(cudaLaunchKernel(fn, dim3(grid), dim3(h->g.threads * hv), args, h->g.smem, h->st));
    return FD_OK;
}

// Steps [k0, k1) with fn: the per-step kernel's groups are steps; the blocked kernel's are the
// blocks that intersect the span, plus the group holding the last block's updates.
// NVTX range around a host call (header-only NVTX v3: free unless a profiler is attached), so that
// a timeline shows the library's phases: set-up, forward launches, adjoint recompute and sweep,
// batches, checkpoints.
namespace {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

static int launch_steps(fd_handle *h, const void *fn, const Inst *d_inst, int k0, int k1, bool adj_groups = false)
{
    NvtxRange r(fn == h->kfwd ? "fd: forward launch" : "fd: adjoint / recompute launch");
    const int tb = h->g.tb;
    if (tb) return launch(h, fn, d_inst, k0 / tb, (k1 + tb - 1) / tb + 1, k0, k1, adj_groups);
    return launch(h, fn, d_inst, k0, k1, k0, k1, adj_groups);
}

// A zero nz (structs initialised before the field existed) means a single plane.
static const fd_problem *normalized(const fd_problem *p, fd_problem &q)
{
    if (!p) return p;
    q = *p;
    if (q.nz == 0) q.nz = 1;
    return &q;
}

static int prepare(const fd_problem *p, Sched &s, Geo &g, size_t *bytes, Layout *Lout, char *ws,
                   Ctrl *ctrl)
{
    int rc = validate(p);
    if (rc) return rc;
    build_schedule(*p, p->max_steps, s);
    make_geo(*p, s, 0, g);
    if (g.tmem_cols > 512) return FD_ERR_INVALID_ARG;  // a CTA's tensor memory holds 512 columns
    // closed loop: a step's per-chunk tallies fit the stage ring (the decider's scratch)
    if (closed_loop(*p) && (size_t)g.maxC * 4 > (size_t)g.NS * g.RS * g.threads * 16) return FD_ERR_INVALID_ARG;
    Carve c(ws);
    Ctrl cc = carve_ctrl(c);
    Layout L;
    carve_instance(c, *p, g, s, L);
    c.take(sizeof(Inst) * 2);                                     // device instance descriptors
    c.take(sizeof(long long) * (size_t)(p->max_steps + 2));       // group offsets
    c.take(sizeof(int2) * (size_t)(p->max_steps + 2));            // group info
    if (adaptive_adjoint(*p)) {                                   // the adjoint's groups
        c.take(sizeof(long long) * (size_t)(p->max_steps + 2));
        c.take(sizeof(int2) * (size_t)(p->max_steps + 2));
    }
    if (bytes) *bytes = c.off;
    if (Lout) *Lout = L;
    if (ctrl) *ctrl = cc;
    return FD_OK;
}

extern "C" {

int fd_weights(double gamma, int64_t n, double *psi, double *dpsi)
{
    if (n < 1 || !psi || !std::isfinite(gamma)) return FD_ERR_INVALID_ARG;
    gl_weights(gamma, n, psi, dpsi);
    return FD_OK;
}

int fd_schedule(const fd_problem *p, int64_t k, int64_t *lags, int64_t *mult, int64_t cap, int64_t *n)
{
    if (!p || k < 0 || !n || (cap > 0 && (!lags || !mult))) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_SHORT && p->mem_L < 1) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_ADAPTIVE && p->mem_a < 2) return FD_ERR_INVALID_ARG;
    if (p->mem_mode < FD_MEM_FULL || p->mem_mode > FD_MEM_ADAPTIVE) return FD_ERR_INVALID_ARG;
    fd_problem q = *p;
    Sched s;
    build_schedule(q, k + 1, s);
    const int4 e = s.step[k];
    int64_t cnt = 0;
    auto put = [&](int64_t lag, int64_t m) {
        if (cnt < cap) {
            lags[cnt] = lag;
            mult[cnt] = m;
        }
        ++cnt;
    };
    put(0, 1);
    for (int i = 1; i <= e.x; ++i) put(i, 1);
    for (int i = 0; i < e.y; ++i) put(s.G[i].lag, s.G[i].mult);
    for (int i = e.z; i <= e.w; ++i) put(i, 1);
    *n = cnt;
    return FD_OK;
}

int fd_workspace_bytes(const fd_problem *p, size_t *bytes)
{
    if (!bytes) return FD_ERR_INVALID_ARG;
    fd_problem q;
    p = normalized(p, q);
    Sched s;
    Geo g;
    return prepare(p, s, g, bytes, nullptr, nullptr, nullptr);
}

int fd_init(const fd_problem *p, void *workspace, size_t ws_bytes, void *cuda_stream, fd_handle **out)
{
    NvtxRange r("fd_init: schedule, tables, workspace layout, uploads");
    if (!out) return FD_ERR_INVALID_ARG;
    fd_problem q;
    p = normalized(p, q);
    *out = nullptr;
    fd_handle *h = new (std::nothrow) fd_handle();
    if (!h) return FD_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = prepare(p, h->s, h->g, &need, nullptr, nullptr, nullptr);
    if (rc) {
        delete h;
        return rc;
    }
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || ws_bytes < need) {
        delete h;
        return FD_ERR_WORKSPACE;
    }
    h->p = *p;
    h->st = (cudaStream_t)cuda_stream;
    h->ws = (char *)workspace;
    h->ws_bytes = ws_bytes;
    prepare(p, h->s, h->g, nullptr, &h->L, h->ws, &h->ctrl);
    {
        Carve c(h->ws);
        carve_ctrl(c);
        Layout tmp;
        carve_instance(c, *p, h->g, h->s, tmp);
        h->d_inst = (Inst *)c.take(sizeof(Inst) * 2);
        h->d_goff = (long long *)c.take(sizeof(long long) * (size_t)(p->max_steps + 2));
        h->d_ginfo = (int2 *)c.take(sizeof(int2) * (size_t)(p->max_steps + 2));
        h->d_agoff = nullptr;
        h->d_aginfo = nullptr;
        if (adaptive_adjoint(*p)) {
            h->d_agoff = (long long *)c.take(sizeof(long long) * (size_t)(p->max_steps + 2));
            h->d_aginfo = (int2 *)c.take(sizeof(int2) * (size_t)(p->max_steps + 2));
        }
    }
    h->ctrl_zero_base = (char *)h->L.arrive;
    h->ctrl_zero_bytes = sizeof(unsigned) * (h->g.npar + 1) * (size_t)h->g.T;
    const bool kahan = p->flags & FD_FLAG_KAHAN;
    h->kfwd = p->time_block ? fdk::kernel_tb(p->time_block, false, p->hist_dtype, h->g.tc)
                            : fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, kahan, false);
    h->kadj = !(p->flags & FD_FLAG_KEEP_TAPE) ? nullptr
              : p->time_block ? fdk::kernel_tb(p->time_block, true, p->hist_dtype)
                              : fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, false, true);
    rc = set_smem_attr(h->kfwd, h->g.smem);
    if (!rc && h->kadj) rc = set_smem_attr(h->kadj, h->g.smem);
    if (!rc) rc = resolve_grid(h->kfwd, h->g);
    if (rc) {
        delete h;
        return rc;
    }
    // group table: group k = step k of instance 0
    // groups: step k (per-step kernel) or block b of time_block steps (blocked kernel)
    const int ngroups = h->g.tb ? h->g.nblocks + 1 : p->max_steps;
    h->goff.resize((size_t)ngroups + 1);
    std::vector<int2> info((size_t)ngroups + 1);
    long long acc = 0;
    for (int k = 0; k < ngroups; ++k) {
        h->goff[k] = acc;
        info[k] = make_int2(0, k);
        acc += h->g.tb ? block_units(*p, h->g, k) : step_units(h->g, h->s.step[k]);
    }
    h->goff[ngroups] = acc;
    info[ngroups] = make_int2(0, ngroups);
    if (h->d_agoff) {  // adjoint of adaptive memory: full memory's units, same group numbering
        const fd_problem pf = full_memory(*p);
        h->agoff.resize((size_t)ngroups + 1);
        long long a2 = 0;
        for (int k = 0; k < ngroups; ++k) {
            h->agoff[k] = a2;
            a2 += h->g.tb ? block_units(pf, h->g, k) : step_units(h->g, full_step(k));
        }
        h->agoff[ngroups] = a2;
    }
    build_tables(*p, h->s, h->g, h->t);
    h->inst_fwd = make_inst(*p, h->g, h->L, false);
    h->inst_adj = (p->flags & FD_FLAG_KEEP_TAPE) ? make_inst(*p, h->g, h->L, true) : h->inst_fwd;
    cudaStream_t st = h->st;
    // zero state, history (ragged padding included), scales and status words, then upload
    const size_t used = (size_t)((char *)h->d_inst - h->ws);
    if (cudaMemsetAsync(h->ws, 0, used, st) != cudaSuccess) rc = FD_ERR_CUDA;
    if (!rc) rc = upload_tables(*p, h->s, h->t, h->L, st);
    if (!rc) rc = upload_tmap(*p, h->g, h->L, h->inst_fwd, st);
    if (!rc && cudaMemcpyAsync(h->d_goff, h->goff.data(), sizeof(long long) * h->goff.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && cudaMemcpyAsync(h->d_ginfo, info.data(), sizeof(int2) * info.size(), cudaMemcpyHostToDevice,
                               st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && h->d_agoff &&
        (cudaMemcpyAsync(h->d_agoff, h->agoff.data(), sizeof(long long) * h->agoff.size(), cudaMemcpyHostToDevice,
                         st) != cudaSuccess ||
         cudaMemcpyAsync(h->d_aginfo, info.data(), sizeof(int2) * info.size(), cudaMemcpyHostToDevice, st) !=
             cudaSuccess))
        rc = FD_ERR_CUDA;
    Inst both[2] = {h->inst_fwd, h->inst_adj};
    if (!rc && cudaMemcpyAsync(h->d_inst, both, sizeof(both), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = FD_ERR_CUDA;
    if (rc) {
        (void)cudaGetLastError();
        delete h;
        return rc;
    }
    h->k = 0;
    h->bad = 0;
    *out = h;
    return FD_OK;
}

int fd_set_state(fd_handle *h, const void *u0)
{
    if (!h || !u0) return FD_ERR_INVALID_ARG;
    const size_t bytes = (size_t)h->p.nx * h->p.ny * h->p.nz * h->g.ss;
    CK(cudaMemcpyAsync(h->L.ubuf[0], u0, bytes, cudaMemcpyDefault, h->st));
    if (h->L.ulo[0]) CK(cudaMemsetAsync(h->L.ulo[0], 0, bytes, h->st));
    if (h->L.ckpt) CK(cudaMemcpyAsync(h->L.ckpt, u0, bytes, cudaMemcpyDefault, h->st));
    CK(cudaMemsetAsync(h->ctrl.err, 0, sizeof(int), h->st));
    CK(cudaMemsetAsync(h->ctrl.nonfinite, 0, sizeof(unsigned), h->st));
    CK(cudaMemsetAsync(h->ctrl.err_info, 0, 8 * sizeof(long long), h->st));
    if (h->L.clD) {
        const size_t K = (size_t)h->p.max_steps;
        CK(cudaMemsetAsync(h->L.clD, 0, K * sizeof(double), h->st));
        CK(cudaMemsetAsync(h->L.clM, 0, K * sizeof(double), h->st));
        CK(cudaMemsetAsync(h->L.clrows, 0, K * sizeof(unsigned), h->st));
        CK(cudaMemsetAsync(h->L.clterms, 0, sizeof(unsigned long long), h->st));
        CK(cudaMemsetAsync(h->L.clword, 0, sizeof(unsigned long long) * (size_t)h->L.clslots * h->g.maxC, h->st));
    }
    h->k = 0;
    h->bad = 0;
    return FD_OK;
}

int fd_step(fd_handle *h, int nsteps)
{
    NvtxRange r("fd_step");
    if (!h || nsteps < 0) return FD_ERR_INVALID_ARG;
    if (h->bad) return FD_ERR_STATE;
    if (h->k + nsteps > h->p.max_steps) return FD_ERR_STATE;
    if (nsteps == 0) return FD_OK;
    const int rc = launch_steps(h, h->kfwd, h->d_inst, (int)h->k, (int)(h->k + nsteps));
    if (rc) return rc;
    h->k += nsteps;
    return FD_OK;
}

int fd_get_state(fd_handle *h, void *u_out)
{
    if (!h || !u_out) return FD_ERR_INVALID_ARG;
    const size_t bytes = (size_t)h->p.nx * h->p.ny * h->p.nz * h->g.ss;
    CK(cudaMemcpyAsync(u_out, h->L.ubuf[h->k & 1], bytes, cudaMemcpyDefault, h->st));
    return FD_OK;
}

int64_t fd_current_step(fd_handle *h) { return h ? h->k : -1; }

int fd_get_status(fd_handle *h)
{
    if (!h) return FD_ERR_INVALID_ARG;
    int err = 0;
    unsigned nf = 0;
    CK(cudaMemcpyAsync(&err, h->ctrl.err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&nf, h->ctrl.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const int s = status_from(err, nf);
    if (s == FD_ERR_TIMEOUT) h->bad = 1;
    return s;
}

int fd_memory_terms(fd_handle *h, int64_t *terms)
{
    if (!h || !terms) return FD_ERR_INVALID_ARG;
    if (h->L.clterms) {
        unsigned long long n = 0;
        CK(cudaMemcpyAsync(&n, h->L.clterms, sizeof(n), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        *terms = (int64_t)n;
        return FD_OK;
    }
    int64_t n = 0;
    for (int64_t k = 0; k < h->k; ++k) n += n_terms(h->s.step[k]) + 1;
    *terms = n;
    return FD_OK;
}

int fd_get_error_info(fd_handle *h, int64_t info[8])
{
    if (!h || !info) return FD_ERR_INVALID_ARG;
    long long v[8];
    CK(cudaMemcpyAsync(v, h->ctrl.err_info, sizeof(v), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < 8; ++i) info[i] = v[i];
    return FD_OK;
}

int fd_run(fd_handle *h, int nsteps, void *u_out)
{
    int rc = fd_step(h, nsteps);
    if (rc) return rc;
    if (u_out) {
        rc = fd_get_state(h, u_out);
        if (rc) return rc;
    }
    return fd_get_status(h);
}

int fd_adjoint(fd_handle *h, const void *dJ_duK, void *dJ_du0, double *dJ_dgamma, double *dJ_dalpha,
               double dJ_dreact[4])
{
    NvtxRange r("fd_adjoint: checkpoint recompute and reverse sweep");
    if (!h || !dJ_duK) return FD_ERR_INVALID_ARG;
    if (!(h->p.flags & FD_FLAG_KEEP_TAPE) || !h->kadj || h->bad || h->k < 1) return FD_ERR_STATE;
    const fd_problem &p = h->p;
    const int K = (int)h->k;
    const int C = p.ckpt_every ? p.ckpt_every : 200;
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
    const size_t ub = (size_t)N * h->g.ss;
    cudaStream_t st = h->st;
    int rc = FD_OK;
    CK(cudaMemcpyAsync(h->L.abuf[0], dJ_duK, ub, cudaMemcpyDefault, st));
    if (h->L.alo[0]) CK(cudaMemsetAsync(h->L.alo[0], 0, ub, st));
    CK(cudaMemsetAsync(h->L.dots, 0, sizeof(double) * 8 * (size_t)h->g.T, st));
    const int nseg = (K + C - 1) / C;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int c = sgi * C, ce = std::min(K, c + C);
        // forward recompute of u^c .. u^{ce-1} into the segment buffer (history rows kept)
        Inst rec = h->inst_fwd;
        rec.ubuf[0] = h->L.rec[0];
        rec.ubuf[1] = h->L.rec[1];
        rec.ulo[0] = h->L.rlo[0];
        rec.ulo[1] = h->L.rlo[1];
        if (rec.ulo[0]) CK(cudaMemsetAsync(h->L.rlo[c & 1], 0, ub, st));
        rec.hist_write = 0;
        rec.stall = 0;
        rec.tape = h->L.seg;
        rec.tape_k0 = c;
        rec.tape_every = 1;
        rec.tape_rows = h->L.seg_rows;
        Inst adj = h->inst_adj;
        adj.uadj_r0 = c;
        adj.adj_K = K;
        CK(cudaMemcpyAsync(&h->d_inst[0], &rec, sizeof(Inst), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(&h->d_inst[1], &adj, sizeof(Inst), cudaMemcpyHostToDevice, st));
        const char *uc = h->L.ckpt + (size_t)sgi * ub;
        CK(cudaMemcpyAsync(h->L.rec[c & 1], uc, ub, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(h->L.seg, uc, ub, cudaMemcpyDeviceToDevice, st));
        if (ce - c > 1) {
            rc = launch_steps(h, h->kfwd, &h->d_inst[0], c, ce - 1);
            if (rc) break;
        }
        // adjoint steps q = K-ce .. K-1-c  (r = K-1-q from ce-1 down to c)
        rc = launch_steps(h, h->kadj, &h->d_inst[1], K - ce, K - c, true);
        if (rc) break;
    }
    // restore the forward descriptor
    Inst both[2] = {h->inst_fwd, h->inst_adj};
    if (cudaMemcpyAsync(h->d_inst, both, sizeof(both), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (rc) return rc;
    std::vector<double> dots((size_t)8 * h->g.T);
    CK(cudaMemcpyAsync(dots.data(), h->L.dots, sizeof(double) * dots.size(), cudaMemcpyDeviceToHost, st));
    if (dJ_du0) CK(cudaMemcpyAsync(dJ_du0, h->L.abuf[K & 1], ub, cudaMemcpyDefault, st));
    const int s = fd_get_status(h);  // synchronises
    if (s) return s;
    double d[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < h->g.T; ++t)
        for (int i = 0; i < 6; ++i) d[i] += dots[(size_t)t * 8 + i];
    const double S = p.alpha * std::pow(p.dt, p.gamma) / (p.dx * p.dx);
    if (dJ_dalpha) *dJ_dalpha = (S / p.alpha) * d[0];
    if (dJ_dgamma) *dJ_dgamma = S * (std::log(p.dt) * d[0] + d[1]);
    if (dJ_dreact)
        for (int i = 0; i < 4; ++i) dJ_dreact[i] = p.dt * d[2 + i];
    return FD_OK;
}

// ------------------------------------------------------------------- checkpoints

namespace {

// Layout of a checkpoint: this header, then u^k, its compensation part (F32 state), the history
// rows 0 .. rows-1 of each plane, the state-precision ring (when separate) and the row scales of
// rows 0 .. rows-1.  rows = min(k, cap) when the history keeps every step, else the whole ring.
struct SaveHeader {
    char magic[8];
    int64_t k, N, ss, comp, cap, pitch, planes, rows, hring_sep, hring_cap, hring_pitch, hscale, T;
    int64_t nx, ny, nz, ndim, max_steps, mem_mode, mem_L, mem_a, rule, time_block, sdt, hdt, adt, flags, bc;
    int64_t closed;  // closed-loop memory: the rows' maxima and counts, and the terms counter follow
    double gamma, alpha, dt, dx, react[4], tau;
};

void save_plan(const fd_handle *h, int64_t k, SaveHeader &hd, size_t &total)
{
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "FDSAVE2", 8);
    const fd_problem &p = h->p;
    const Geo &g = h->g;
    hd.k = k;
    hd.N = (int64_t)p.nx * p.ny * p.nz;
    hd.ss = g.ss;
    hd.comp = h->L.ulo[0] ? 1 : 0;
    hd.cap = g.cap;
    hd.pitch = g.pitch;
    hd.planes = g.lo_plane ? 2 : 1;
    hd.rows = (g.cap >= p.max_steps) ? std::min<int64_t>(k, g.cap) : g.cap;
    hd.hring_sep = g.hring_sep;
    hd.hring_cap = g.hring_sep ? g.hring_cap : 0;
    hd.hring_pitch = g.hring_sep ? g.hring_pitch : 0;
    hd.hscale = h->L.hscale ? 1 : 0;
    hd.T = g.T;
    hd.nx = p.nx;
    hd.ny = p.ny;
    hd.nz = p.nz;
    hd.ndim = p.ndim;
    hd.max_steps = p.max_steps;
    hd.mem_mode = p.mem_mode;
    hd.mem_L = p.mem_L;
    hd.mem_a = p.mem_a;
    hd.rule = p.adaptive_rule;
    hd.time_block = p.time_block;
    hd.sdt = p.state_dtype;
    hd.hdt = p.hist_dtype;
    hd.adt = p.accum_dtype;
    hd.flags = p.flags;
    hd.bc = p.bc;
    hd.gamma = p.gamma;
    hd.alpha = p.alpha;
    hd.dt = p.dt;
    hd.dx = p.dx;
    for (int i = 0; i < 4; ++i) hd.react[i] = p.react[i];
    hd.closed = h->L.clD ? 1 : 0;
    hd.tau = hd.closed ? p.mem_tau : 0.0;
    total = sizeof(SaveHeader) + (size_t)hd.N * hd.ss * (1 + hd.comp) + (size_t)(hd.planes * hd.rows * hd.pitch) +
            (size_t)(hd.hring_cap * hd.hring_pitch) + (size_t)(hd.hscale * hd.rows * hd.T) * sizeof(float) +
            (size_t)hd.closed * ((size_t)k * (2 * sizeof(double) + sizeof(unsigned)) + sizeof(unsigned long long) +
                                 (size_t)h->L.clslots * (h->L.clgmax + sizeof(unsigned long long) * g.maxC));
}

// The pieces of a checkpoint in order: (device address, bytes).
std::vector<std::pair<char *, size_t>> save_pieces(const fd_handle *h, const SaveHeader &hd)
{
    std::vector<std::pair<char *, size_t>> v;
    const size_t ub = (size_t)hd.N * hd.ss;
    v.emplace_back(h->L.ubuf[hd.k & 1], ub);
    if (hd.comp) v.emplace_back(h->L.ulo[hd.k & 1], ub);
    for (int64_t pl = 0; pl < hd.planes; ++pl)
        v.emplace_back(h->L.hist + (size_t)(pl * hd.cap * hd.pitch), (size_t)(hd.rows * hd.pitch));
    if (hd.hring_cap) v.emplace_back(h->L.hring, (size_t)(hd.hring_cap * hd.hring_pitch));
    if (hd.hscale) v.emplace_back(reinterpret_cast<char *>(h->L.hscale), (size_t)(hd.rows * hd.T) * sizeof(float));
    if (hd.closed) {
        v.emplace_back(reinterpret_cast<char *>(h->L.clD), (size_t)hd.k * sizeof(double));
        v.emplace_back(reinterpret_cast<char *>(h->L.clM), (size_t)hd.k * sizeof(double));
        v.emplace_back(reinterpret_cast<char *>(h->L.clrows), (size_t)hd.k * sizeof(unsigned));
        v.emplace_back(reinterpret_cast<char *>(h->L.clterms), sizeof(unsigned long long));
        // the decisions already made for the steps after k (by rows before k)
        v.emplace_back(reinterpret_cast<char *>(h->L.clcnt), (size_t)h->L.clslots * h->L.clgmax);
        v.emplace_back(reinterpret_cast<char *>(h->L.clword), sizeof(unsigned long long) * (size_t)h->L.clslots * h->g.maxC);
    }
    return v;
}

}  // namespace

int fd_save_bytes(fd_handle *h, size_t *bytes)
{
    if (!h || !bytes) return FD_ERR_INVALID_ARG;
    if (h->p.flags & FD_FLAG_KEEP_TAPE) return FD_ERR_UNSUPPORTED;
    SaveHeader hd;
    save_plan(h, h->k, hd, *bytes);
    return FD_OK;
}

int fd_save(fd_handle *h, void *buf, size_t bytes)
{
    NvtxRange r("fd_save");
    if (!h || !buf) return FD_ERR_INVALID_ARG;
    if (h->p.flags & FD_FLAG_KEEP_TAPE) return FD_ERR_UNSUPPORTED;
    if (h->bad) return FD_ERR_STATE;
    SaveHeader hd;
    size_t total = 0;
    save_plan(h, h->k, hd, total);
    if (bytes < total) return FD_ERR_INVALID_ARG;
    char *out = static_cast<char *>(buf);
    CK(cudaMemcpyAsync(out, &hd, sizeof(hd), cudaMemcpyDefault, h->st));
    size_t off = sizeof(hd);
    for (const auto &pc : save_pieces(h, hd)) {
        if (pc.second) CK(cudaMemcpyAsync(out + off, pc.first, pc.second, cudaMemcpyDefault, h->st));
        off += pc.second;
    }
    CK(cudaStreamSynchronize(h->st));  // (the header copy reads a host stack variable)
    return FD_OK;
}

int fd_load(fd_handle *h, const void *buf, size_t bytes)
{
    NvtxRange r("fd_load");
    if (!h || !buf || bytes < sizeof(SaveHeader)) return FD_ERR_INVALID_ARG;
    if (h->p.flags & FD_FLAG_KEEP_TAPE) return FD_ERR_UNSUPPORTED;
    SaveHeader in;
    CK(cudaMemcpy(&in, buf, sizeof(in), cudaMemcpyDefault));
    if (std::memcmp(in.magic, "FDSAVE2", 8) || in.k < 0 || in.k > h->p.max_steps) return FD_ERR_INVALID_ARG;
    SaveHeader hd;
    size_t total = 0;
    save_plan(h, in.k, hd, total);
    if (std::memcmp(&in, &hd, sizeof(hd)) || bytes < total) return FD_ERR_INVALID_ARG;  // another problem
    const char *src = static_cast<const char *>(buf);
    size_t off = sizeof(hd);
    for (const auto &pc : save_pieces(h, hd)) {
        if (pc.second) CK(cudaMemcpyAsync(pc.first, src + off, pc.second, cudaMemcpyDefault, h->st));
        off += pc.second;
    }
    if (hd.closed && in.k < h->p.max_steps) {  // rows from k on: not yet written (the handle may have run further)
        const size_t rest = (size_t)(h->p.max_steps - in.k);
        CK(cudaMemsetAsync(h->L.clD + in.k, 0, rest * sizeof(double), h->st));
        CK(cudaMemsetAsync(h->L.clM + in.k, 0, rest * sizeof(double), h->st));
        CK(cudaMemsetAsync(h->L.clrows + in.k, 0, rest * sizeof(unsigned), h->st));
    }
    CK(cudaMemsetAsync(h->ctrl.err, 0, sizeof(int), h->st));
    CK(cudaMemsetAsync(h->ctrl.nonfinite, 0, sizeof(unsigned), h->st));
    CK(cudaMemsetAsync(h->ctrl.err_info, 0, 8 * sizeof(long long), h->st));
    CK(cudaStreamSynchronize(h->st));
    h->k = in.k;
    h->bad = 0;
    return FD_OK;
}

int fd_get_geometry(fd_handle *h, fd_geometry *g)
{
    if (!h || !g) return FD_ERR_INVALID_ARG;
    g->tile_threads = h->g.threads;
    g->tile_points = h->g.P;
    g->tiles = h->g.T;
    g->chunk_terms = h->g.R;
    g->stage_rows = h->g.RS;
    g->stages = h->g.NS;
    g->ctas_per_sm = h->g.ctas;
    g->grid = h->g.grid;
    g->head_lags = h->g.head;
    g->units_total = h->goff.back();
    int64_t rows = 0;
    for (const int4 &e : h->s.step) rows += n_terms(e);
    const int64_t N = (int64_t)h->p.nx * h->p.ny * h->p.nz;
    g->hist_rows_total = rows;
    g->terms_total = (rows + (int64_t)h->s.step.size()) * N;
    g->time_block = h->g.tb;
    g->block_updates = h->g.ub;
    g->far_tensor_cores = h->g.tc;
    g->smem_bytes = (int64_t)h->g.smem;
    g->head_rows_total = 0;
    g->stream_rows_total = h->g.tb ? blocked_stream_rows(h->p, h->g, &g->head_rows_total) : rows;
    return FD_OK;
}

int fd_destroy(fd_handle *h)
{
    delete h;
    return FD_OK;
}

const char *fd_strerror(int code)
{
    switch (code) {
    case FD_OK: return "ok";
    case FD_ERR_INVALID_ARG: return "invalid argument";
    case FD_ERR_UNSTABLE: return "S exceeds the explicit stability bound 2^gamma/(4 ndim)";
    case FD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FD_ERR_CUDA: return "CUDA runtime error";
    case FD_ERR_NONFINITE: return "non-finite value in the state";
    case FD_ERR_TIMEOUT: return "device-side wait timed out";
    case FD_ERR_STATE: return "call out of order for this handle";
    case FD_ERR_UNSUPPORTED: return "unsupported dtype / mode combination";
    default: return "unknown error";
    }
}

}  // extern "C"

// =================================================================== batches

struct fd_batch {
    std::vector<fd_problem> p;
    cudaStream_t st;
    char *ws;
    std::vector<Geo> g;
    std::vector<Sched> s;
    std::vector<Tables> t;
    std::vector<Layout> L;
    Ctrl ctrl;
    unsigned *counters;
    size_t counter_bytes;
    Inst *d_inst;
    long long *d_goff;
    int2 *d_ginfo;
    std::vector<long long> goff;
    std::vector<int2> ginfo;
    const void *kfn;
    int threads, RS, NS, grid, rmax, tb;
    size_t smem, smem_half;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

int batch_plan(const fd_problem *probs_in, int count, fd_batch &b, size_t *bytes, char *ws)
{
    if (!probs_in || count < 1) return FD_ERR_INVALID_ARG;
    std::vector<fd_problem> norm(probs_in, probs_in + count);
    for (fd_problem &q : norm)
        if (q.nz == 0) q.nz = 1;
    const fd_problem *probs = norm.data();
    for (int i = 0; i < count; ++i) {
        const int rc = validate(&probs[i]);
        if (rc) return rc;
        if (probs[i].state_dtype != probs[0].state_dtype || probs[i].hist_dtype != probs[0].hist_dtype ||
            probs[i].accum_dtype != probs[0].accum_dtype ||
            ((probs[i].flags ^ probs[0].flags) & (FD_FLAG_KAHAN | FD_FLAG_KEEP_TAPE)))
            return FD_ERR_INVALID_ARG;
        if (probs[i].flags & (FD_FLAG_KEEP_TAPE | FD_FLAG_CLOSED_LOOP)) return FD_ERR_UNSUPPORTED;
        if (probs[i].time_block != probs[0].time_block) return FD_ERR_INVALID_ARG;  // one kernel per batch
    }
    b.p.assign(probs, probs + count);
    b.s.resize(count);
    b.g.resize(count);
    b.L.resize(count);
    const int threads = probs[0].tile_threads ? probs[0].tile_threads : 256;
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        build_schedule(probs[i], probs[i].max_steps, b.s[i]);
        make_geo(probs[i], b.s[i], threads, b.g[i]);
        if (b.g[i].tmem_cols > 512) return FD_ERR_INVALID_ARG;  // a CTA's tensor memory holds 512 columns
        tiles += b.g[i].T;
    }
    // the launch's threads per (half-)CTA: the instances' resolved tile width (the tensor-core
    // kernels fix it by history type and block length), the same for every instance
    for (int i = 1; i < count; ++i)
        if (b.g[i].threads != b.g[0].threads || b.g[i].fsub != b.g[0].fsub || b.g[i].RS != b.g[0].RS)
            return FD_ERR_INVALID_ARG;
    b.threads = b.g[0].threads;
    b.RS = b.g[0].RS;
    b.NS = b.g[0].NS;
    b.rmax = 0;
    for (int i = 0; i < count; ++i) b.rmax = std::max(b.rmax, b.g[i].tb ? b.g[i].rwin : b.g[i].R);
    b.tb = probs[0].time_block;
    b.smem_half = b.g[0].tc ? smem_half_tc(b.g[0], b.rmax, probs[0].hist_dtype != FD_BF16) : 0;
    b.smem = b.g[0].tc ? b.g[0].halves * b.smem_half + 1024
             : b.tb    ? smem_bytes_tb(b.g[0], b.rmax, probs[0].hist_dtype == FD_F16)
                       : smem_bytes(b.g[0], b.rmax);
    Carve c(ws);
    b.ctrl = carve_ctrl(c);
    int64_t counters = 0;
    for (int i = 0; i < count; ++i) counters += (int64_t)(b.g[i].npar + 1) * b.g[i].T;
    b.counter_bytes = sizeof(unsigned) * (size_t)counters;
    b.counters = (unsigned *)c.take(b.counter_bytes);
    int64_t toff = 0;
    for (int i = 0; i < count; ++i) {
        unsigned *cnt = b.counters ? b.counters + toff : nullptr;
        carve_instance(c, probs[i], b.g[i], b.s[i], b.L[i], cnt, true);
        toff += (b.g[i].npar + 1) * (int64_t)b.g[i].T;
    }
    // groups: step-major (per-step kernel) or block-major (blocked kernel: group b of an
    // instance holds its block b's far units and block b-1's updates), then instance
    int maxK = 0, maxB = 0;
    for (int i = 0; i < count; ++i) {
        maxK = std::max(maxK, probs[i].max_steps);
        maxB = std::max(maxB, b.g[i].nblocks);
    }
    b.goff.clear();
    b.ginfo.clear();
    long long acc = 0;
    if (b.tb) {
        for (int k = 0; k <= maxB; ++k)
            for (int i = 0; i < count; ++i) {
                if (k > b.g[i].nblocks) continue;
                b.goff.push_back(acc);
                b.ginfo.push_back(make_int2(i, k));
                acc += block_units(probs[i], b.g[i], k);
            }
    } else {
        for (int k = 0; k < maxK; ++k)
            for (int i = 0; i < count; ++i) {
                if (k >= probs[i].max_steps) continue;
                b.goff.push_back(acc);
                b.ginfo.push_back(make_int2(i, k));
                acc += step_units(b.g[i], b.s[i].step[k]);
            }
    }
    b.goff.push_back(acc);
    b.ginfo.push_back(make_int2(0, 0));
    b.d_inst = (Inst *)c.take(sizeof(Inst) * (size_t)count);
    b.d_goff = (long long *)c.take(sizeof(long long) * b.goff.size());
    b.d_ginfo = (int2 *)c.take(sizeof(int2) * b.ginfo.size());
    if (bytes) *bytes = c.off;
    return FD_OK;
}

}  // namespace

extern "C" {

int fd_batch_workspace_bytes(const fd_problem *probs, int count, size_t *bytes)
{
    if (!bytes) return FD_ERR_INVALID_ARG;
    fd_batch b;
    return batch_plan(probs, count, b, bytes, nullptr);
}

int fd_batch_init(const fd_problem *probs, int count, void *workspace, size_t ws_bytes, void *cuda_stream,
                  fd_batch **out)
{
    if (!out) return FD_ERR_INVALID_ARG;
    *out = nullptr;
    fd_batch *b = new (std::nothrow) fd_batch();
    if (!b) return FD_ERR_INVALID_ARG;
    b->graph = nullptr;
    b->exec = nullptr;
    size_t need = 0;
    int rc = batch_plan(probs, count, *b, &need, nullptr);
    if (!rc && (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || ws_bytes < need))
        rc = FD_ERR_WORKSPACE;
    if (!rc) rc = batch_plan(probs, count, *b, nullptr, (char *)workspace);
    if (rc) {
        delete b;
        return rc;
    }
    b->ws = (char *)workspace;
    b->st = (cudaStream_t)cuda_stream;
    const bool kahan = b->p[0].flags & FD_FLAG_KAHAN;
    b->kfn = b->tb ? fdk::kernel_tb(b->tb, false, b->p[0].hist_dtype, b->g[0].tc)
                   : fdk::kernel_for(b->p[0].state_dtype, b->p[0].hist_dtype, b->p[0].accum_dtype, kahan, false);
    Geo g0 = b->g[0];
    g0.smem = b->smem;  // the launch's shared memory: the largest chunk over the instances
    rc = set_smem_attr(b->kfn, b->smem);
    if (!rc) rc = resolve_grid(b->kfn, g0);
    b->grid = g0.grid;
    cudaStream_t st = b->st;
    const size_t used = (size_t)((char *)b->d_inst - b->ws);
    if (!rc && cudaMemsetAsync(b->ws, 0, used, st) != cudaSuccess) rc = FD_ERR_CUDA;
    b->t.resize(count);
    std::vector<Inst> insts(count);
    for (int i = 0; i < count && !rc; ++i) {
        build_tables(b->p[i], b->s[i], b->g[i], b->t[i]);
        rc = upload_tables(b->p[i], b->s[i], b->t[i], b->L[i], st);
        insts[i] = make_inst(b->p[i], b->g[i], b->L[i], false);
        if (!rc) rc = upload_tmap(b->p[i], b->g[i], b->L[i], insts[i], st);
    }
    if (!rc && cudaMemcpyAsync(b->d_inst, insts.data(), sizeof(Inst) * insts.size(), cudaMemcpyHostToDevice,
                               st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && cudaMemcpyAsync(b->d_goff, b->goff.data(), sizeof(long long) * b->goff.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && cudaMemcpyAsync(b->d_ginfo, b->ginfo.data(), sizeof(int2) * b->ginfo.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FD_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = FD_ERR_CUDA;
    // graph: clear control words and counters, then the persistent kernel
    if (!rc) {
        Launch L;
        std::memset(&L, 0, sizeof(L));
        L.inst = b->d_inst;
        L.g_off = b->d_goff;
        L.g_info = b->d_ginfo;
        L.g_begin = 0;
        L.g_end = (int)b->goff.size() - 1;
        L.k0 = 0;
        L.k_end = 0x7fffffff;  // blocked kernel: each instance stops at its own step count
        L.stage_rows = b->RS;
        L.stages = b->NS;
        L.rmax = b->rmax;
        L.smem_half = (int)b->smem_half;
        L.fsub = b->g[0].fsub;
        L.nm_tc = b->g[0].nmtc;
        L.queue = b->ctrl.queue;
        L.err = b->ctrl.err;
        L.nonfinite = b->ctrl.nonfinite;
        L.err_info = b->ctrl.err_info;
        L.timeout_ns = (long long)(b->p[0].timeout_ms ? b->p[0].timeout_ms : 10000) * 1000000LL;
        cudaGraphNode_t m1, m2, kn;
        cudaMemsetParams mp;
        std::memset(&mp, 0, sizeof(mp));
        mp.dst = b->ctrl.queue;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 256 / 4;  // queue, err and nonfinite share the 256-byte control block
        mp.height = 1;
        cudaMemsetParams mc = mp;
        mc.dst = b->counters;
        mc.width = b->counter_bytes / 4;
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof(kp));
        void *args[] = {&L};
        kp.func = (void *)b->kfn;
        const int hv = b->g[0].halves;
        kp.gridDim = dim3((unsigned)((std::min<long long>(b->grid, b->goff.back()) + hv - 1) / hv));
        kp.blockDim = dim3(b->threads * hv);
        kp.sharedMemBytes = (unsigned)b->smem;
        kp.kernelParams = args;
        if (cudaGraphCreate(&b->graph, 0) != cudaSuccess ||
            cudaGraphAddMemsetNode(&m1, b->graph, nullptr, 0, &mp) != cudaSuccess ||
            cudaGraphAddMemsetNode(&m2, b->graph, &m1, 1, &mc) != cudaSuccess ||
            cudaGraphAddKernelNode(&kn, b->graph, &m2, 1, &kp) != cudaSuccess ||
            cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
            rc = FD_ERR_CUDA;
    }
    if (rc) {
        (void)cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return rc;
    }
    *out = b;
    return FD_OK;
}

int fd_batch_set_state(fd_batch *b, int i, const void *u0)
{
    if (!b || !u0 || i < 0 || i >= (int)b->p.size()) return FD_ERR_INVALID_ARG;
    const size_t bytes = (size_t)b->p[i].nx * b->p[i].ny * b->p[i].nz * b->g[i].ss;
    CK(cudaMemcpyAsync(b->L[i].ubuf[0], u0, bytes, cudaMemcpyDefault, b->st));
    if (b->L[i].ulo[0]) CK(cudaMemsetAsync(b->L[i].ulo[0], 0, bytes, b->st));
    return FD_OK;
}

int fd_batch_run(fd_batch *b)
{
    NvtxRange r("fd_batch_run: graph launch");
    if (!b) return FD_ERR_INVALID_ARG;
    CK(cudaGraphLaunch(b->exec, b->st));
    return FD_OK;
}

int fd_batch_get_state(fd_batch *b, int i, void *u_out)
{
    if (!b || !u_out || i < 0 || i >= (int)b->p.size()) return FD_ERR_INVALID_ARG;
    const size_t bytes = (size_t)b->p[i].nx * b->p[i].ny * b->p[i].nz * b->g[i].ss;
    CK(cudaMemcpyAsync(u_out, b->L[i].ubuf[b->p[i].max_steps & 1], bytes, cudaMemcpyDefault, b->st));
    return FD_OK;
}

int fd_batch_get_status(fd_batch *b)
{
    if (!b) return FD_ERR_INVALID_ARG;
    int err = 0;
    unsigned nf = 0;
    CK(cudaMemcpyAsync(&err, b->ctrl.err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    CK(cudaMemcpyAsync(&nf, b->ctrl.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, b->st));
    CK(cudaStreamSynchronize(b->st));
    return status_from(err, nf);
}

int fd_batch_get_geometry(fd_batch *b, int i, fd_geometry *g)
{
    if (!b || !g || i < 0 || i >= (int)b->p.size()) return FD_ERR_INVALID_ARG;
    const Geo &q = b->g[i];
    g->tile_threads = q.threads;
    g->tile_points = q.P;
    g->tiles = q.T;
    g->chunk_terms = q.R;
    g->stage_rows = b->RS;
    g->stages = b->NS;
    g->ctas_per_sm = b->grid / std::max(1, device_sms());
    g->grid = b->grid;
    g->head_lags = q.head;
    int64_t units = 0, rows = 0;
    for (const int4 &e : b->s[i].step) {
        units += step_units(q, e);
        rows += n_terms(e);
    }
    if (q.tb) {
        units = 0;
        for (int64_t k = 0; k <= q.nblocks; ++k) units += block_units(b->p[i], q, k);
    }
    const int64_t N = (int64_t)b->p[i].nx * b->p[i].ny * b->p[i].nz;
    g->units_total = units;
    g->hist_rows_total = rows;
    g->terms_total = (rows + (int64_t)b->s[i].step.size()) * N;
    g->head_rows_total = 0;
    g->stream_rows_total = q.tb ? blocked_stream_rows(b->p[i], q, &g->head_rows_total) : rows;
    g->time_block = q.tb;
    g->block_updates = q.ub;
    g->far_tensor_cores = q.tc;
    g->smem_bytes = (int64_t)b->smem;
    return FD_OK;
}

int fd_batch_destroy(fd_batch *b)
{
    if (!b) return FD_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return FD_OK;
}

int fd_run_batch(const fd_problem *probs, int count, void *const *u_io, void *workspace, size_t ws_bytes,
                 void *cuda_stream)
{
    if (!u_io) return FD_ERR_INVALID_ARG;
    fd_batch *b = nullptr;
    int rc = fd_batch_init(probs, count, workspace, ws_bytes, cuda_stream, &b);
    if (rc) return rc;
    for (int i = 0; i < count && !rc; ++i) rc = fd_batch_set_state(b, i, u_io[i]);
    if (!rc) rc = fd_batch_run(b);
    for (int i = 0; i < count && !rc; ++i) rc = fd_batch_get_state(b, i, u_io[i]);
    if (!rc) rc = fd_batch_get_status(b);
    fd_batch_destroy(b);
    return rc;
}

}  // extern "C"

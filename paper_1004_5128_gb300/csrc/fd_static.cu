// fd_static.cu -- fd_run_static: a forward run whose scratch lives in a static device array.
//
// Some callers cannot allocate device memory: a plugin embedded in a host application that
// owns the GPU's allocator and hands the plugin only a stream, or a control loop that is not
// allowed to allocate once it has started.  For them this file provides one entry point that
// allocates nothing -- no cudaMalloc/cudaFree, no allocating library routine, and no host heap
// either.  It runs the same persistent engine kernel as fd_run, with every piece of scratch
// memory (state double buffer, delta history, partial sums, counters, weight and schedule
// tables) carved from fd_static_scratch, a file-scope array of FD_STATIC_SCRATCH_BYTES that
// every GPU loading the library holds until the process exits.  The caller passes only the
// input u0 and the output buffer.
//
// The weight, schedule and work-group tables are computed on the device by a one-thread set-up
// kernel with the same arithmetic as the host tables of fd_init (FP64 recurrence for psi,
// rounded once), so for equal launch geometry the result equals fd_run's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/fd.h"
#include "fd_kernels.h"

using fdk::Inst;
using fdk::Launch;

// The shared scratch of fd_run_static (host code must use its device address, see below).
static __device__ __align__(256) unsigned char fd_static_scratch[FD_STATIC_SCRATCH_BYTES];

namespace {

// The host-side name fd_static_scratch is only a stand-in: ask the runtime for the array's
// address on the current device.  This is done on every call, with the caller's device current,
// and never cached: after cudaDeviceReset or a release of the primary context the module is
// loaded again, possibly at another address.  Once the module is loaded the lookup is cheap.
int scratch_address(char **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, fd_static_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    *out = static_cast<char *>(p);
    return FD_OK;
}

inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int esize(int d) { return d == FD_F64 ? 8 : d == FD_F32 ? 4 : (d == FD_BF16 || d == FD_F16) ? 2 : 0; }

// Bump carve over the static array; returns nullptr once past the end.
struct Carve {
    char *base;
    size_t off, cap;
    char *take(size_t bytes)
    {
        off = up(off, 256);
        char *p = base + off;
        off += up(bytes, 256);
        return off <= cap ? p : nullptr;
    }
};

int check_problem(const fd_problem *p, int nsteps)
{
    if (!p || nsteps < 0) return FD_ERR_INVALID_ARG;
    if (p->ndim < 1 || p->ndim > 3) return FD_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->ndim == 1 && p->ny != 1) || (p->ndim < 3 && p->nz != 1))
        return FD_ERR_INVALID_ARG;
    if ((int64_t)p->nx * p->ny * p->nz > (int64_t)1 << 30) return FD_ERR_INVALID_ARG;
    if (!(p->gamma > 0.0 && p->gamma < 2.0) || !(p->alpha > 0.0) || !(p->dt > 0.0) || !(p->dx > 0.0))
        return FD_ERR_INVALID_ARG;
    for (double r : p->react)
        if (!std::isfinite(r)) return FD_ERR_INVALID_ARG;
    if (p->bc != FD_BC_DIRICHLET0 && p->bc != FD_BC_NOFLUX) return FD_ERR_INVALID_ARG;
    if (p->mem_mode < FD_MEM_FULL || p->mem_mode > FD_MEM_ADAPTIVE) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_SHORT && p->mem_L < 1) return FD_ERR_INVALID_ARG;
    if (p->mem_mode == FD_MEM_ADAPTIVE &&
        (p->mem_a < 2 || (p->adaptive_rule != FD_ADAPT_PAPER && p->adaptive_rule != FD_ADAPT_PARTITION)))
        return FD_ERR_INVALID_ARG;
    if (p->timeout_ms < 0 || p->head_lags < 0 || p->head_lags > 4096) return FD_ERR_INVALID_ARG;
    if (p->tile_threads && (p->tile_threads < 32 || p->tile_threads > 512 || p->tile_threads % 32))
        return FD_ERR_INVALID_ARG;
    if (p->chunk_terms < 0 || p->stage_rows < 0 || p->stage_rows > 64 || p->stages < 0 || p->stages > 16 ||
        p->ctas_per_sm < 0 || p->ctas_per_sm > 8)
        return FD_ERR_INVALID_ARG;
    if (p->flags & FD_FLAG_KEEP_TAPE) return FD_ERR_UNSUPPORTED;  // forward only
    if (p->flags & FD_FLAG_CLOSED_LOOP) return FD_ERR_UNSUPPORTED;  // open-loop schedules only
    if (p->time_block) return FD_ERR_UNSUPPORTED;                 // per-step kernel only
    if (!fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, p->flags & FD_FLAG_KAHAN, false))
        return FD_ERR_UNSUPPORTED;
    if (!(p->flags & FD_FLAG_ALLOW_UNSTABLE)) {
        const double S = p->alpha * std::pow(p->dt, p->gamma) / (p->dx * p->dx);
        if (S > std::pow(2.0, p->gamma) / (4.0 * p->ndim) * (1.0 + 1e-12)) return FD_ERR_UNSTABLE;
    }
    return FD_OK;
}

// Tables the set-up kernel writes (all inside the static array).
struct Tabs {
    int mode, L, a, rule, K, T, R, head, acc64;
    double gamma;
    double *psid;       // FP64 weights, K+1
    char *psi;          // weights in the accumulator type, K+1
    int4 *sched;        // K
    int *glag;          // medians, up to K
    char *gcoef;
    long long *gend;
    long long *goff;    // K+1
    int2 *ginfo;        // K+1
};

__device__ void put_acc(char *dst, int i, double v, int acc64)
{
    if (acc64) reinterpret_cast<double *>(dst)[i] = v;
    else reinterpret_cast<float *>(dst)[i] = (float)v;
}

// One thread: psi by the recurrence of Section 2.1, the adaptive medians of Proposition 3.1
// (literal or partition reading), the per-step schedule and the work-group offsets.
__global__ void static_tables_kernel(const Tabs t)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double prev = 1.0;
    t.psid[0] = 1.0;
    put_acc(t.psi, 0, 1.0, t.acc64);
    for (int m = 1; m <= t.K; ++m) {
        const double f = __ddiv_rn(__dadd_rn(__dadd_rn((double)m, -2.0), t.gamma), (double)m);
        prev = __dmul_rn(prev, f);
        t.psid[m] = prev;
        put_acc(t.psi, m, prev, t.acc64);
    }
    int ng = 0;
    if (t.mode == FD_MEM_ADAPTIVE) {
        const long long kmax = t.K, a = t.a;
        if (t.rule == FD_ADAPT_PAPER) {
            long long lo = a;
            bool done = false;
            for (long long i = 2; !done && lo + 1 <= kmax; ++i) {
                const long long hi = (lo > (long long)4e15 / a) ? (long long)4e15 : lo * a;
                const long long d = 2 * i - 1;
                for (long long m = lo + i; m <= hi; m += d) {
                    if (m + i - 1 > kmax) {
                        done = true;
                        break;
                    }
                    t.glag[ng] = (int)m;
                    t.gend[ng] = m + i - 1;
                    put_acc(t.gcoef, ng, __dmul_rn((double)d, t.psid[m]), t.acc64);
                    ++ng;
                }
                lo = hi;
            }
        } else {
            long long c = a + 1, hi = a;
            bool done = false;
            for (long long i = 2; !done; ++i) {
                hi = (hi > (long long)4e15 / a) ? (long long)4e15 : hi * a;
                const long long d = 2 * i - 1;
                for (long long m = c + i - 1; m <= hi; m = c + i - 1) {
                    if (c + d - 1 > kmax) {
                        done = true;
                        break;
                    }
                    t.glag[ng] = (int)m;
                    t.gend[ng] = c + d - 1;
                    put_acc(t.gcoef, ng, __dmul_rn((double)d, t.psid[m]), t.acc64);
                    ++ng;
                    c += d;
                }
            }
        }
    }
    int g = 0;
    long long off = 0;
    for (int k = 0; k < t.K; ++k) {
        int4 e = make_int4(0, 0, 1, 0);
        if (t.mode == FD_MEM_FULL) {
            e.x = k;
        } else if (t.mode == FD_MEM_SHORT) {
            e.x = min(t.L, k);
        } else if (k <= t.a) {
            e.x = k;
        } else {
            e.x = t.a;
            while (g < ng && t.gend[g] <= k) ++g;
            e.y = g;
            e.z = (int)((g ? t.gend[g - 1] : t.a) + 1);
            e.w = k;
        }
        t.sched[k] = e;
        const long long n = (long long)e.x + e.y + (e.w >= e.z ? e.w - e.z + 1 : 0) - min(t.head, e.x);
        t.goff[k] = off;
        t.ginfo[k] = make_int2(0, k);
        off += (long long)t.T * max(1LL, (n + t.R - 1) / t.R);
    }
    t.goff[t.K] = off;
    t.ginfo[t.K] = make_int2(0, t.K);
}

}  // namespace

extern "C" int fd_run_static(const fd_problem *p_in, const void *u0, int nsteps, void *u_out, void *cuda_stream)
{
    fd_problem q;  // a zero nz (structs initialised before the field existed) means one plane
    if (p_in) {
        q = *p_in;
        if (q.nz == 0) q.nz = 1;
    }
    const fd_problem *p = p_in ? &q : nullptr;
    int rc = check_problem(p, nsteps);
    if (rc) return rc;
    if (!u0 || !u_out) return FD_ERR_INVALID_ARG;
    char *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    // every step takes at least 48 bytes of tables (weights, schedule, group offsets): longer runs
    // cannot fit, and rejecting them here keeps the size arithmetic below far from overflow
    if ((int64_t)nsteps * 48 > (int64_t)FD_STATIC_SCRATCH_BYTES) return FD_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const int sh = esize(p->hist_dtype), ss = esize(p->state_dtype), sa = esize(p->accum_dtype);
    const size_t ubytes = (size_t)N * ss;
    if (nsteps == 0) {
        if (cudaMemcpyAsync(u_out, u0, ubytes, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            (void)cudaGetLastError();
            return FD_ERR_CUDA;
        }
        return FD_OK;
    }

    // launch geometry (the same rules as fd_init, with the chunk count bounded by n(k) <= k)
    const int K = nsteps, V = 16 / sh;
    int th = p->tile_threads;
    if (!th) {
        th = 256;
        while (th > 64 && (N + V - 1) / V <= th / 2) th /= 2;
    }
    const int P = th * V;
    const int T = (int)((N + P - 1) / P);
    const int RS = p->stage_rows ? p->stage_rows : 8, NS = p->stages ? p->stages : 3;
    int cap = K;
    if (p->mem_mode == FD_MEM_SHORT) cap = std::min(p->mem_L + 1, K);
    cap = std::max(cap, 1);
    const bool hsep = p->hist_dtype != p->state_dtype;
    int head = p->head_lags ? p->head_lags : (hsep ? 32 : 8);
    if (!hsep && cap < head + 1) head = std::max(1, cap - 1);
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    int ctas = p->ctas_per_sm ? p->ctas_per_sm : 2;
    int R = p->chunk_terms;
    if (!R) {
        int64_t r = ((int64_t)(K - 1) * T + 4LL * sms * ctas - 1) / (4LL * sms * ctas);
        r = std::min<int64_t>(std::max<int64_t>(r, 2 * RS), 256);
        R = (int)((r + RS - 1) / RS * RS);
    }
    const int maxC = std::max(1, (K - 1 + R - 1) / R);
    const int64_t pitch = (int64_t)up((size_t)N * sh, 256);
    const int64_t hpitch = hsep ? (int64_t)up(up((size_t)N, 8) * ss, 256) : pitch;
    const int64_t ppitch = (int64_t)up(up((size_t)N, 8) * sa, 256);
    const size_t smem = (size_t)NS * RS * th * 16 + (size_t)R * (2 * sa + 4) + 32 + 8 * (size_t)NS;
    const bool comp = p->state_dtype == FD_F32 && !(p->flags & FD_FLAG_PLAIN_STATE);

    // carve the static scratch; a problem that does not fit is rejected
    Carve c{base, 0, FD_STATIC_SCRATCH_BYTES};
    char *ctrl = c.take(256);
    const int npar = 4;
    unsigned *cnt = (unsigned *)c.take(sizeof(unsigned) * (npar + 1) * (size_t)T);
    char *ub0 = c.take(ubytes), *ub1 = c.take(ubytes);
    char *lo0 = comp ? c.take(ubytes) : base, *lo1 = comp ? c.take(ubytes) : base;
    char *hist = c.take((size_t)cap * pitch);
    char *hring = hsep ? c.take((size_t)(head + 1) * hpitch) : hist;
    float *hscale = (p->hist_dtype == FD_F16) ? (float *)c.take((size_t)cap * T * sizeof(float)) : nullptr;
    char *part = c.take((size_t)npar * maxC * ppitch);
    Tabs t;
    t.mode = p->mem_mode;
    t.L = p->mem_L;
    t.a = p->mem_a;
    t.rule = p->adaptive_rule;
    t.K = K;
    t.T = T;
    t.R = R;
    t.head = head;
    t.acc64 = (sa == 8);
    t.gamma = p->gamma;
    t.psid = (double *)c.take(sizeof(double) * (size_t)(K + 1));
    t.psi = c.take((size_t)sa * (K + 1));
    t.sched = (int4 *)c.take(sizeof(int4) * (size_t)K);
    t.glag = (int *)c.take(sizeof(int) * (size_t)K);
    t.gcoef = c.take((size_t)sa * K);
    t.gend = (long long *)c.take(sizeof(long long) * (size_t)K);
    t.goff = (long long *)c.take(sizeof(long long) * (size_t)(K + 1));
    t.ginfo = (int2 *)c.take(sizeof(int2) * (size_t)(K + 1));
    Inst *d_inst = (Inst *)c.take(sizeof(Inst));
    if (!d_inst || c.off > FD_STATIC_SCRATCH_BYTES) return FD_ERR_WORKSPACE;  // beyond the static maximum
    if (smem + 4096 > (size_t)optin) return FD_ERR_INVALID_ARG;

    Inst I;
    std::memset(&I, 0, sizeof(I));
    I.ndim = p->ndim;
    I.nx = p->nx;
    I.ny = p->ny;
    I.bc = p->bc;
    I.N = (int)N;
    I.nz = p->nz;
    I.T = T;
    I.P = P;
    I.R = R;
    I.hist_write = 1;
    I.cap = cap;
    I.maxC = maxC;
    I.npar = npar;
    I.stall = (p->flags & FD_FLAG_INJECT_STALL) ? 1 : 0;
    I.head = head;
    I.hring_cap = hsep ? head + 1 : cap;
    I.hring_sep = hsep ? 1 : 0;
    I.tape_every = 1;
    I.S = p->alpha * std::pow(p->dt, p->gamma) / (p->dx * p->dx);
    I.dt = p->dt;
    for (int i = 0; i < 4; ++i) I.react[i] = p->react[i];
    I.pitch = pitch;
    I.part_pitch = ppitch;
    I.hring_pitch = hpitch;
    I.hring = hring;
    I.hist = hist;
    I.hscale = hscale;
    I.ubuf[0] = ub0;
    I.ubuf[1] = ub1;
    I.ulo[0] = comp ? lo0 : nullptr;
    I.ulo[1] = comp ? lo1 : nullptr;
    I.part = part;
    I.arrive = cnt;
    I.done = cnt + npar * T;
    I.psi = t.psi;
    I.sched = t.sched;
    I.g_lag = t.glag;
    I.g_coef = t.gcoef;

    const void *fn = fdk::kernel_for(p->state_dtype, p->hist_dtype, p->accum_dtype, p->flags & FD_FLAG_KAHAN, false);
    int occ = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 4096) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, th, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    if (occ < 1) return FD_ERR_INVALID_ARG;
    ctas = std::min(ctas, occ);

    Launch L;
    std::memset(&L, 0, sizeof(L));
    L.inst = d_inst;
    L.g_off = t.goff;
    L.g_info = t.ginfo;
    L.g_begin = 0;
    L.g_end = K;
    L.k0 = 0;
    L.stage_rows = RS;
    L.stages = NS;
    L.rmax = R;
    L.queue = (unsigned long long *)ctrl;
    L.err = (int *)(ctrl + 64);
    L.nonfinite = (unsigned *)(ctrl + 128);
    L.err_info = (long long *)(ctrl + 192);
    L.timeout_ns = (long long)(p->timeout_ms ? p->timeout_ms : 10000) * 1000000LL;

    // the array keeps the previous call's contents: clear what must start at zero
    bool ok = cudaMemsetAsync(ctrl, 0, 256, st) == cudaSuccess &&
              cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (npar + 1) * (size_t)T, st) == cudaSuccess &&
              (!comp || cudaMemsetAsync(lo0, 0, ubytes, st) == cudaSuccess) &&
              cudaMemcpyAsync(d_inst, &I, sizeof(I), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(ub0, u0, ubytes, cudaMemcpyDefault, st) == cudaSuccess;
    if (ok) {
        static_tables_kernel<<<1, 32, 0, st>>>(t);
        ok = cudaGetLastError() == cudaSuccess;
    }
    void *args[] = {&L};
    if (ok)
        ok = cudaLaunchKernel(fn, dim3(sms * ctas), dim3(th), args, smem, st) == cudaSuccess &&
             cudaMemcpyAsync(u_out, K & 1 ? ub1 : ub0, ubytes, cudaMemcpyDefault, st) == cudaSuccess;
    int err = 0;
    unsigned nf = 0;
    if (ok)
        ok = cudaMemcpyAsync(&err, L.err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaMemcpyAsync(&nf, L.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return FD_ERR_CUDA;
    }
    if (err) return FD_ERR_TIMEOUT;
    if (nf) return FD_ERR_NONFINITE;
    return FD_OK;
}

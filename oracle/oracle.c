/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * A direct restatement of the explicit Grunwald-Letnikov scheme of Sprouse,
 * MacDonald & Silva: weights by the recurrence of Section 2.1, the FTCS
 * stencil of eq. deltasimp, the update of eq. frac_final, the short memory of
 * eq. frac_shortmemory and the adaptive memory of Definitions 3.1/3.2 and
 * Proposition 3.1.  Plain loops, double precision, ascending-lag Neumaier
 * summation.  The only reordering is across grid points (each point's own
 * sum keeps the ascending-lag order), which changes no result.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- helpers */

/* Neumaier's improvement of Kahan summation: s += x with running error c. */
static inline void nadd(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

static int check_problem(const or_problem *p, long K)
{
    if (!p || K < 0) return -1;
    if (p->ndim < 1 || p->ndim > 3) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->ndim == 1 && p->ny != 1) || (p->ndim < 3 && p->nz != 1))
        return -1;
    if (p->bc != OR_BC_DIRICHLET0 && p->bc != OR_BC_NOFLUX) return -1;
    if (!(p->dt > 0) || !(p->dx > 0)) return -1;
    if (p->mem_mode == OR_MEM_SHORT && p->mem_L < 0) return -1;
    if (p->mem_mode == OR_MEM_ADAPTIVE && p->mem_a < 2) return -1;
    if (p->mem_mode < OR_MEM_FULL || p->mem_mode > OR_MEM_ADAPTIVE) return -1;
    return 0;
}

/* Five-point (2-D) / three-point (1-D) unnormalised difference of eq. deltasimp:
 *   delta_{j,l} = u_{j+1,l} + u_{j-1,l} - 4 u_{j,l} + u_{j,l+1} + u_{j,l-1}.
 * Ghost values outside the grid: 0 (Dirichlet, "edge set to zero", Section 3.1)
 * or the boundary cell's own value (no-flux, cell-centred mirror). */
static void apply_L(const or_problem *p, const double *u, double *out)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long pl = (long)nx * ny; /* points per z-plane */
    const int mirror = (p->bc == OR_BC_NOFLUX);
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long i = (long)z * pl + (long)y * nx + x;
                const double c = u[i];
                const double g = mirror ? c : 0.0;
                const double r = (x + 1 < nx) ? u[i + 1] : g;
                const double l = (x > 0) ? u[i - 1] : g;
                if (p->ndim == 1) {
                    out[i] = r - 2.0 * c + l;
                } else if (p->ndim == 2) {
                    const double up = (y + 1 < ny) ? u[i + nx] : g;
                    const double dn = (y > 0) ? u[i - nx] : g;
                    out[i] = r + l - 4.0 * c + up + dn;
                } else {
                    /* the 7-point analogue of eq. deltasimp: x pair, -6 u, y pair, z pair */
                    const double up = (y + 1 < ny) ? u[i + nx] : g;
                    const double dn = (y > 0) ? u[i - nx] : g;
                    const double fw = (z + 1 < nz) ? u[i + pl] : g;
                    const double bk = (z > 0) ? u[i - pl] : g;
                    out[i] = r + l - 6.0 * c + up + dn + fw + bk;
                }
            }
        }
    }
}

/* Transpose of apply_L, written in scatter form from the rows of L: row i
 * reads each in-grid neighbour with weight 1 (a ghost reads nothing under
 * Dirichlet, or u_i itself under the mirror rule) and u_i with weight -2 ndim;
 * L^T v sends v_i back to every column that row i read. */
static void apply_LT(const or_problem *p, const double *v, double *out)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long pl = (long)nx * ny;
    const int mirror = (p->bc == OR_BC_NOFLUX);
    const long N = pl * nz;
    memset(out, 0, sizeof(double) * (size_t)N);
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long i = (long)z * pl + (long)y * nx + x;
                const double vi = v[i];
                const int ndir = 2 * p->ndim;
                const long nb[6] = {x + 1 < nx ? i + 1 : -1, x > 0 ? i - 1 : -1,
                                    y + 1 < ny ? i + nx : -1, y > 0 ? i - nx : -1,
                                    z + 1 < nz ? i + pl : -1, z > 0 ? i - pl : -1};
                for (int d = 0; d < ndir; ++d) {
                    if (nb[d] >= 0)
                        out[nb[d]] += vi;
                    else if (mirror)
                        out[i] += vi;
                }
                out[i] += -2.0 * p->ndim * vi;
            }
        }
    }
}

static double react_f(const double r[4], double u)
{
    return r[0] + u * (r[1] + u * (r[2] + u * r[3]));
}

static double react_df(const double r[4], double u)
{
    return r[1] + u * (2.0 * r[2] + u * 3.0 * r[3]);
}

/* ------------------------------------------------------------------ weights */

int or_weights(double gamma, long n, double *psi, double *dpsi)
{
    if (n < 1 || !psi) return -1;
    psi[0] = 1.0; /* psi(g, 0) = 1 */
    if (dpsi) dpsi[0] = 0.0;
    for (long m = 1; m < n; ++m) {
        /* psi(g, m) = -psi(g, m-1) (2 - g - m) / m */
        psi[m] = -psi[m - 1] * (2.0 - gamma - (double)m) / (double)m;
        /* d/dg of the same product: the factor -(2-g-m)/m has derivative 1/m */
        if (dpsi)
            dpsi[m] = -dpsi[m - 1] * (2.0 - gamma - (double)m) / (double)m + psi[m - 1] / (double)m;
    }
    return 0;
}

/* ----------------------------------------------------------------- schedule */

static long ipow_capped(long a, long e, long cap)
{
    long r = 1;
    for (long i = 0; i < e; ++i) {
        if (r > cap / a) return cap + 1;
        r *= a;
    }
    return r;
}

long or_schedule(int mem_mode, long L, long a, int rule, long k, long *lag, long *mult)
{
    if (k < 0 || !lag || !mult) return -1;
    long n = 0;
    if (mem_mode == OR_MEM_FULL || (mem_mode == OR_MEM_ADAPTIVE && k <= a)) {
        /* eq. frac_final: m = 0..k; adaptive with k inside the base interval [0, a] */
        for (long m = 0; m <= k; ++m) { lag[n] = m; mult[n] = 1; ++n; }
        return n;
    }
    if (mem_mode == OR_MEM_SHORT) {
        if (L < 0) return -1;
        const long top = L < k ? L : k; /* eq. frac_shortmemory: m = 0..min(L/dt, k) */
        for (long m = 0; m <= top; ++m) { lag[n] = m; mult[n] = 1; ++n; }
        return n;
    }
    if (mem_mode != OR_MEM_ADAPTIVE || a < 2) return -1;

    /* Base interval [0, a]: every lag, weight 1 (first sum of eq. eq:adapttime). */
    for (long m = 0; m <= a; ++m) { lag[n] = m; mult[n] = 1; ++n; }
    long e = a; /* last lag covered so far */
    if (rule == OR_ADAPT_PAPER) {
        /* Intervals I_i = [a^{i-1} + i, a^i], i >= 2 (Definition 3.1), sampled at the
         * medians m_i = a^{i-1} + (2i-1) eta - i + 1, eta = 1, 2, ... (Proposition 3.1),
         * each weighted by its increment length d = 2i-1 (Definition 3.2).  A median m
         * stands for lags m-(i-1) .. m+(i-1); a block is used while it ends at or
         * before k, and the tail sum covers e+1 .. k. */
        for (long i = 2;; ++i) {
            const long lo = ipow_capped(a, i - 1, k + 1); /* a^{i-1} */
            if (lo + 1 > k) break;
            const long hi = ipow_capped(a, i, 4 * k + 4);   /* a^i */
            const long d = 2 * i - 1;
            int stop = 0;
            for (long eta = 1;; ++eta) {
                const long m = lo + d * eta - i + 1;
                if (m > hi) break;
                if (m + i - 1 > k) { stop = 1; break; }
                lag[n] = m; mult[n] = d; ++n;
                e = m + i - 1;
            }
            if (stop) break;
        }
    } else if (rule == OR_ADAPT_PARTITION) {
        /* Same intervals and spacings, but consecutive increments of width d_i tile
         * the lags from a+1 onward exactly once (a cursor replaces the fixed
         * interval origin): medians stay in I_i while m <= a^i. */
        long c = a + 1; /* first uncovered lag */
        int stop = 0;
        for (long i = 2; !stop; ++i) {
            const long hi = ipow_capped(a, i, 4 * k + 4);
            const long d = 2 * i - 1;
            if (c + d - 1 > k) break;
            for (;;) {
                const long m = c + i - 1;
                if (m > hi) break;
                if (c + d - 1 > k) { stop = 1; break; }
                lag[n] = m; mult[n] = d; ++n;
                c += d;
            }
        }
        e = c - 1;
    } else {
        return -1;
    }
    /* Tail: lags e+1 .. k, every point, weight 1 (last sum of eq. eq:adapttime). */
    for (long m = e + 1; m <= k; ++m) { lag[n] = m; mult[n] = 1; ++n; }
    return n;
}

/* ------------------------------------------------------------------ forward */

static long history_rows(const or_problem *p, long K)
{
    long cap = K;
    if (p->mem_mode == OR_MEM_SHORT && (long)p->mem_L + 1 < K) cap = (long)p->mem_L + 1;
    return cap < 1 ? 1 : cap;
}

int or_run(const or_problem *p, const double *u0, long K, double *uK, double *tape, int threads)
{
    if (check_problem(p, K) || !u0 || !uK) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    const long cap = history_rows(p, K);
    const double S = p->alpha * pow(p->dt, p->gamma) / (p->dx * p->dx);

    double *psi = malloc(sizeof(double) * (size_t)(K + 1));
    double *hist = malloc(sizeof(double) * (size_t)cap * (size_t)N);
    double *u = malloc(sizeof(double) * (size_t)N);
    double *un = malloc(sizeof(double) * (size_t)N);
    double *sum = malloc(sizeof(double) * (size_t)N);
    double *cmp = malloc(sizeof(double) * (size_t)N);
    long *lag = malloc(sizeof(long) * (size_t)(K + 1));
    long *mult = malloc(sizeof(long) * (size_t)(K + 1));
    double *coef = malloc(sizeof(double) * (size_t)(K + 1));
    if (!psi || !hist || !u || !un || !sum || !cmp || !lag || !mult || !coef) {
        free(psi); free(hist); free(u); free(un); free(sum); free(cmp); free(lag); free(mult);
        free(coef);
        return -2;
    }
    or_weights(p->gamma, K + 1, psi, NULL);
    memcpy(u, u0, sizeof(double) * (size_t)N);
    if (tape) memcpy(tape, u, sizeof(double) * (size_t)N);
#ifdef _OPENMP
    const int nthr = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
    const long BLK = 512;
    const long nblk = (N + BLK - 1) / BLK;

    for (long k = 0; k < K; ++k) {
        apply_L(p, u, hist + (size_t)(k % cap) * (size_t)N); /* delta^k */
        const long n = or_schedule(p->mem_mode, p->mem_L, p->mem_a, p->adaptive_rule, k, lag, mult);
        for (long t = 0; t < n; ++t) coef[t] = (double)mult[t] * psi[lag[t]];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
        for (long b = 0; b < nblk; ++b) {
            const long j0 = b * BLK, j1 = (j0 + BLK < N) ? j0 + BLK : N;
            for (long j = j0; j < j1; ++j) { sum[j] = 0.0; cmp[j] = 0.0; }
            for (long t = 0; t < n; ++t) { /* ascending lag */
                const double *row = hist + (size_t)((k - lag[t]) % cap) * (size_t)N;
                const double c = coef[t];
                for (long j = j0; j < j1; ++j) nadd(&sum[j], &cmp[j], c * row[j]);
            }
            for (long j = j0; j < j1; ++j) {
                /* eq. frac_final with f outside the memory sum:
                 * u^{k+1} = u^k + dt f(u^k) + S sum_m c_m delta^{k-m} */
                un[j] = u[j] + p->dt * react_f(p->react, u[j]) + S * (sum[j] + cmp[j]);
            }
        }
        double *tmp = u; u = un; un = tmp;
        if (tape) memcpy(tape + (size_t)(k + 1) * (size_t)N, u, sizeof(double) * (size_t)N);
    }
    memcpy(uK, u, sizeof(double) * (size_t)N);
    free(psi); free(hist); free(u); free(un); free(sum); free(cmp); free(lag); free(mult); free(coef);
    return 0;
}

/* ------------------------------------------------ BF16-stored history forward */

double or_round_bf16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    const double f = frexp(x, &e); /* x = f 2^e, 0.5 <= |f| < 1: 8 significant bits = f 2^8 */
    return ldexp(nearbyint(ldexp(f, 8)), e - 8);
}

int or_run_bf16(const or_problem *p, const double *u0, long K, long blk, long head, double *uK, int threads)
{
    if (check_problem(p, K) || !u0 || !uK || blk < 0 || head < 0) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    const long cap = history_rows(p, K);
    const double S = p->alpha * pow(p->dt, p->gamma) / (p->dx * p->dx);

    double *psi = malloc(sizeof(double) * (size_t)(K + 1));
    double *hist = malloc(sizeof(double) * (size_t)cap * (size_t)N);  /* delta as computed */
    double *hist16 = malloc(sizeof(double) * (size_t)cap * (size_t)N); /* its BF16 rounding */
    double *u = malloc(sizeof(double) * (size_t)N);
    double *un = malloc(sizeof(double) * (size_t)N);
    long *lag = malloc(sizeof(long) * (size_t)(K + 1));
    long *mult = malloc(sizeof(long) * (size_t)(K + 1));
    if (!psi || !hist || !hist16 || !u || !un || !lag || !mult) {
        free(psi); free(hist); free(hist16); free(u); free(un); free(lag); free(mult);
        return -2;
    }
    or_weights(p->gamma, K + 1, psi, NULL);
    memcpy(u, u0, sizeof(double) * (size_t)N);
#ifdef _OPENMP
    const int nthr = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
    for (long k = 0; k < K; ++k) {
        double *row = hist + (size_t)(k % cap) * (size_t)N;
        apply_L(p, u, row); /* delta^k */
        for (long j = 0; j < N; ++j) hist16[(size_t)(k % cap) * (size_t)N + j] = or_round_bf16(row[j]);
        const long n = or_schedule(p->mem_mode, p->mem_L, p->mem_a, p->adaptive_rule, k, lag, mult);
        const long w = head + (blk > 0 ? k % blk : 0); /* lags <= w as computed */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
        for (long j = 0; j < N; ++j) {
            double sum = 0.0, cmp = 0.0;
            for (long t = 0; t < n; ++t) { /* ascending lag */
                const double *h = (lag[t] <= w ? hist : hist16) + (size_t)((k - lag[t]) % cap) * (size_t)N;
                nadd(&sum, &cmp, (double)mult[t] * psi[lag[t]] * h[j]);
            }
            /* eq. frac_final with f outside the memory sum */
            un[j] = u[j] + p->dt * react_f(p->react, u[j]) + S * (sum + cmp);
        }
        double *tmp = u; u = un; un = tmp;
    }
    memcpy(uK, u, sizeof(double) * (size_t)N);
    free(psi); free(hist); free(hist16); free(u); free(un); free(lag); free(mult);
    return 0;
}

/* ------------------------------------------------ closed-loop adaptive memory */

int or_run_closed(const or_problem *p, const double *u0, long K, double tau, double *uK, long *nterms,
                  double *margin, int threads)
{
    if (check_problem(p, K) || !u0 || !uK || p->mem_mode != OR_MEM_ADAPTIVE || !(tau >= 0.0)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    const double S = p->alpha * pow(p->dt, p->gamma) / (p->dx * p->dx);
    double *psi = malloc(sizeof(double) * (size_t)(K + 1));
    double *hist = malloc(sizeof(double) * (size_t)K * (size_t)N);
    double *D = calloc((size_t)K, sizeof(double)); /* D_r: largest change from row r-1 to row r */
    double *M = calloc((size_t)K, sizeof(double)); /* M_r: largest |delta^r| */
    double *u = malloc(sizeof(double) * (size_t)N);
    double *un = malloc(sizeof(double) * (size_t)N);
    long *lag = malloc(sizeof(long) * (size_t)(K + 1));
    long *mult = malloc(sizeof(long) * (size_t)(K + 1));
    /* the step's terms after the feedback: a median, or its increment's lags one by one */
    long *tl = malloc(sizeof(long) * (size_t)(K + 1) * 2);
    double *tc = malloc(sizeof(double) * (size_t)(K + 1) * 2);
    if (!psi || !hist || !D || !M || !u || !un || !lag || !mult || !tl || !tc) {
        free(psi); free(hist); free(D); free(M); free(u); free(un); free(lag); free(mult); free(tl); free(tc);
        return -2;
    }
    or_weights(p->gamma, K + 1, psi, NULL);
    memcpy(u, u0, sizeof(double) * (size_t)N);
#ifdef _OPENMP
    const int nthr = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
    long total = 0;
    double mg = INFINITY; /* closest decision to the threshold, relative to it */
    for (long k = 0; k < K; ++k) {
        double *row = hist + (size_t)k * (size_t)N;
        apply_L(p, u, row); /* delta^k */
        for (long j = 0; j < N; ++j) {
            M[k] = fmax(M[k], fabs(row[j]));
            if (k) D[k] = fmax(D[k], fabs(row[j] - row[(long)j - N]));
        }
        const long n = or_schedule(p->mem_mode, p->mem_L, p->mem_a, p->adaptive_rule, k, lag, mult);
        long nt = 0;
        for (long t = 0; t < n; ++t) {
            const long m = lag[t], d = mult[t];
            if (d == 1) {
                tl[nt] = m; tc[nt] = psi[m]; ++nt;
                continue;
            }
            const long h = (d - 1) / 2, lo = m - h, hi = m + h; /* the increment's lags */
            double var = 0.0;
            for (long r = k - hi + 1; r <= k - lo; ++r) var += D[r];
            const double ref = M[k - m];
            const int smooth = isinf(tau) || ((ref > 0.0) ? (var / ref < tau) : (var == 0.0 && tau > 0.0));
            if (!isinf(tau) && tau > 0.0 && ref > 0.0) mg = fmin(mg, fabs(var / ref - tau) / tau);
            if (smooth) {
                tl[nt] = m; tc[nt] = (double)d * psi[m]; ++nt;
            } else {
                for (long l = lo; l <= hi; ++l) { tl[nt] = l; tc[nt] = psi[l]; ++nt; }
            }
        }
        total += nt;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
        for (long j = 0; j < N; ++j) {
            double sum = 0.0, cmp = 0.0;
            for (long t = 0; t < nt; ++t) nadd(&sum, &cmp, tc[t] * hist[(size_t)(k - tl[t]) * (size_t)N + j]);
            /* eq. frac_final with f outside the memory sum */
            un[j] = u[j] + p->dt * react_f(p->react, u[j]) + S * (sum + cmp);
        }
        double *tmp = u; u = un; un = tmp;
    }
    memcpy(uK, u, sizeof(double) * (size_t)N);
    if (nterms) *nterms = total;
    if (margin) *margin = mg;
    free(psi); free(hist); free(D); free(M); free(u); free(un); free(lag); free(mult); free(tl); free(tc);
    return 0;
}

/* ------------------------------------------------------ complex-step forward */

static void apply_L_cs(const or_problem *p, const double complex *u, double complex *out)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long pl = (long)nx * ny;
    const int mirror = (p->bc == OR_BC_NOFLUX);
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const long i = (long)z * pl + (long)y * nx + x;
                const double complex c = u[i];
                const double complex g = mirror ? c : 0.0;
                const double complex r = (x + 1 < nx) ? u[i + 1] : g;
                const double complex l = (x > 0) ? u[i - 1] : g;
                if (p->ndim == 1) {
                    out[i] = r - 2.0 * c + l;
                } else if (p->ndim == 2) {
                    const double complex up = (y + 1 < ny) ? u[i + nx] : g;
                    const double complex dn = (y > 0) ? u[i - nx] : g;
                    out[i] = r + l - 4.0 * c + up + dn;
                } else {
                    const double complex up = (y + 1 < ny) ? u[i + nx] : g;
                    const double complex dn = (y > 0) ? u[i - nx] : g;
                    const double complex fw = (z + 1 < nz) ? u[i + pl] : g;
                    const double complex bk = (z > 0) ? u[i - pl] : g;
                    out[i] = r + l - 6.0 * c + up + dn + fw + bk;
                }
            }
        }
    }
}

int or_run_cs(const or_problem *p, double gamma_im, double alpha_im, const double react_im[4],
              const double *u0_re, const double *u0_im, long K, double *uK_re, double *uK_im)
{
    if (check_problem(p, K) || !u0_re || !uK_re || !uK_im) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    const long cap = history_rows(p, K);
    const double complex gam = p->gamma + I * gamma_im;
    const double complex alp = p->alpha + I * alpha_im;
    double complex r[4];
    for (int i = 0; i < 4; ++i) r[i] = p->react[i] + I * (react_im ? react_im[i] : 0.0);
    const double complex S = alp * cpow(p->dt, gam) / (p->dx * p->dx);

    double complex *psi = malloc(sizeof(double complex) * (size_t)(K + 1));
    double complex *hist = malloc(sizeof(double complex) * (size_t)cap * (size_t)N);
    double complex *u = malloc(sizeof(double complex) * (size_t)N);
    double complex *un = malloc(sizeof(double complex) * (size_t)N);
    long *lag = malloc(sizeof(long) * (size_t)(K + 1));
    long *mult = malloc(sizeof(long) * (size_t)(K + 1));
    if (!psi || !hist || !u || !un || !lag || !mult) {
        free(psi); free(hist); free(u); free(un); free(lag); free(mult);
        return -2;
    }
    psi[0] = 1.0;
    for (long m = 1; m <= K; ++m) psi[m] = -psi[m - 1] * (2.0 - gam - (double)m) / (double)m;
    for (long j = 0; j < N; ++j) u[j] = u0_re[j] + I * (u0_im ? u0_im[j] : 0.0);

    for (long k = 0; k < K; ++k) {
        apply_L_cs(p, u, hist + (size_t)(k % cap) * (size_t)N);
        const long n = or_schedule(p->mem_mode, p->mem_L, p->mem_a, p->adaptive_rule, k, lag, mult);
        for (long j = 0; j < N; ++j) {
            double complex s = 0.0;
            for (long t = 0; t < n; ++t)
                s += ((double)mult[t] * psi[lag[t]]) * hist[(size_t)((k - lag[t]) % cap) * (size_t)N + j];
            const double complex f = r[0] + u[j] * (r[1] + u[j] * (r[2] + u[j] * r[3]));
            un[j] = u[j] + p->dt * f + S * s;
        }
        double complex *tmp = u; u = un; un = tmp;
    }
    for (long j = 0; j < N; ++j) { uK_re[j] = creal(u[j]); uK_im[j] = cimag(u[j]); }
    free(psi); free(hist); free(u); free(un); free(lag); free(mult);
    return 0;
}

/* ------------------------------------------------------------------ adjoint */

int or_adjoint(const or_problem *p, const double *u0, long K, const double *target,
               double *J, double *dJ_du0, double *dJ_dgamma, double *dJ_dalpha,
               double dJ_dreact[4], int threads)
{
    if (check_problem(p, K) || !u0 || !target || K < 1) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    const double S = p->alpha * pow(p->dt, p->gamma) / (p->dx * p->dx);
    double *tape = malloc(sizeof(double) * (size_t)(K + 1) * (size_t)N);
    double *lam = malloc(sizeof(double) * (size_t)(K + 1) * (size_t)N); /* lambda^r at row r */
    double *psi = malloc(sizeof(double) * (size_t)(K + 1));
    double *dpsi = malloc(sizeof(double) * (size_t)(K + 1));
    double *g = malloc(sizeof(double) * (size_t)N);
    double *gp = malloc(sizeof(double) * (size_t)N);
    double *du = malloc(sizeof(double) * (size_t)N);
    double *ltg = malloc(sizeof(double) * (size_t)N);
    double *uK = malloc(sizeof(double) * (size_t)N);
    /* adaptive memory: wt[k * K + m] = multiplicity of lag m in step k's schedule */
    int *wt = (p->mem_mode == OR_MEM_ADAPTIVE) ? calloc((size_t)K * (size_t)K, sizeof(int)) : NULL;
    long *slag = (p->mem_mode == OR_MEM_ADAPTIVE) ? malloc(sizeof(long) * (size_t)(K + 1)) : NULL;
    long *smul = (p->mem_mode == OR_MEM_ADAPTIVE) ? malloc(sizeof(long) * (size_t)(K + 1)) : NULL;
    int rc = 0;
    if (!tape || !lam || !psi || !dpsi || !g || !gp || !du || !ltg || !uK ||
        (p->mem_mode == OR_MEM_ADAPTIVE && (!wt || !slag || !smul))) {
        rc = -2;
        goto done;
    }
    if (wt)
        for (long k = 0; k < K; ++k) {
            const long n = or_schedule(p->mem_mode, p->mem_L, p->mem_a, p->adaptive_rule, k, slag, smul);
            if (n < 0) { rc = -1; goto done; }
            for (long t = 0; t < n; ++t) wt[(size_t)k * (size_t)K + (size_t)slag[t]] += (int)smul[t];
        }
    rc = or_run(p, u0, K, uK, tape, threads);
    if (rc) goto done;
    or_weights(p->gamma, K + 1, psi, dpsi);

    double Js = 0.0, Jc = 0.0;
    double *lK = lam + (size_t)K * (size_t)N;
    for (long j = 0; j < N; ++j) {
        const double e = tape[(size_t)K * (size_t)N + j] - target[j];
        lK[j] = e; /* lambda^K = dJ/du^K */
        nadd(&Js, &Jc, 0.5 * e * e);
    }
    double ds[6] = {0}, dc[6] = {0};
#ifdef _OPENMP
    const int nthr = threads > 0 ? threads : omp_get_max_threads();
#endif
    for (long r = K - 1; r >= 0; --r) {
        /* m = 0 .. K-1-r, within the short window m <= L */
        const long nm = (p->mem_mode == OR_MEM_SHORT && p->mem_L < K - 1 - r) ? p->mem_L : K - 1 - r;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
        for (long j = 0; j < N; ++j) {
            double s = 0, c = 0, sp = 0, cp = 0;
            for (long m = 0; m <= nm; ++m) {
                const double l = lam[(size_t)(r + 1 + m) * (size_t)N + j];
                if (wt) { /* delta^r enters step r+m with weight w_{r+m}(m) psi_m */
                    const int w = wt[(size_t)(r + m) * (size_t)K + (size_t)m];
                    if (!w) continue;
                    nadd(&s, &c, ((double)w * psi[m]) * l);
                    nadd(&sp, &cp, ((double)w * dpsi[m]) * l);
                } else {
                    nadd(&s, &c, psi[m] * l);
                    nadd(&sp, &cp, dpsi[m] * l);
                }
            }
            g[j] = s + c;
            gp[j] = sp + cp;
        }
        const double *ur = tape + (size_t)r * (size_t)N;
        const double *l1 = lam + (size_t)(r + 1) * (size_t)N;
        apply_L(p, ur, du); /* delta^r */
        for (long j = 0; j < N; ++j) {
            nadd(&ds[0], &dc[0], du[j] * g[j]);
            nadd(&ds[1], &dc[1], du[j] * gp[j]);
            double pw = 1.0;
            for (int i = 0; i < 4; ++i) {
                nadd(&ds[2 + i], &dc[2 + i], l1[j] * pw);
                pw *= ur[j];
            }
        }
        apply_LT(p, g, ltg);
        double *lr = lam + (size_t)r * (size_t)N;
        for (long j = 0; j < N; ++j)
            lr[j] = l1[j] + p->dt * react_df(p->react, ur[j]) * l1[j] + S * ltg[j];
    }
    if (J) *J = Js + Jc;
    if (dJ_du0) memcpy(dJ_du0, lam, sizeof(double) * (size_t)N);
    const double d0 = ds[0] + dc[0], d1 = ds[1] + dc[1];
    if (dJ_dalpha) *dJ_dalpha = (S / p->alpha) * d0;
    if (dJ_dgamma) *dJ_dgamma = S * (log(p->dt) * d0 + d1);
    if (dJ_dreact)
        for (int i = 0; i < 4; ++i) dJ_dreact[i] = p->dt * (ds[2 + i] + dc[2 + i]);
done:
    free(tape); free(lam); free(psi); free(dpsi); free(g); free(gp);
    free(du); free(ltg); free(uK); free(wt); free(slag); free(smul);
    return rc;
}

/* ------------------------------------------------------ scalar eigenmode run */

int or_scalar_mode(double gamma, double alpha, double dt, double dx, double r1, double Lambda,
                   int mem_mode, long L, long a, int rule, double A0, long K, double *out)
{
    if (K < 0 || !out || !(dt > 0) || !(dx > 0)) return -1;
    const double S = alpha * pow(dt, gamma) / (dx * dx);
    double *psi = malloc(sizeof(double) * (size_t)(K + 1));
    long *lag = malloc(sizeof(long) * (size_t)(K + 1));
    long *mult = malloc(sizeof(long) * (size_t)(K + 1));
    if (!psi || !lag || !mult) { free(psi); free(lag); free(mult); return -2; }
    or_weights(gamma, K + 1, psi, NULL);
    out[0] = A0;
    for (long k = 0; k < K; ++k) {
        const long n = or_schedule(mem_mode, L, a, rule, k, lag, mult);
        if (n < 0) { free(psi); free(lag); free(mult); return -1; }
        double s = 0, c = 0;
        for (long t = 0; t < n; ++t) nadd(&s, &c, ((double)mult[t] * psi[lag[t]]) * out[k - lag[t]]);
        /* delta^r = -Lambda A^r for the mode, so S sum c delta = -S Lambda sum c A */
        out[k + 1] = out[k] + dt * r1 * out[k] - S * Lambda * (s + c);
    }
    free(psi); free(lag); free(mult);
    return 0;
}

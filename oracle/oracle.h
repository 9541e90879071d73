/*
 * FP64 CPU oracle for the explicit Grunwald-Letnikov scheme of the fractional
 * reaction-diffusion equation d^g u/dt^g = alpha Lap u + f(u)
 * (Sprouse, MacDonald & Silva, "Computational Efficiency of Fractional
 * Diffusion Using Adaptive Time Step Memory").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct restatement of the paper's scheme that the CUDA path is checked
 * against.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and it never calls it.
 *
 * Every routine works in double precision (or double complex for the
 * complex-step variant).  Sums over the memory terms run in ascending lag
 * order with Neumaier compensated summation.
 *
 * Pins (checked by the test suite against mathematics, not against this
 * code): closed-form binomial weights, gamma=1 reduces to FTCS heat,
 * single Laplacian eigenmodes reduce to a scalar recursion whose generating
 * function is known, the N=1 relaxation tracks its Mittag-Leffler solution,
 * mass balance under no-flux boundaries, mode coincidence, hand-derived
 * adaptive schedules, a dense linear solve on tiny grids, and finite
 * differences / complex step for the adjoint.
 */
#ifndef FRD_ORACLE_H
#define FRD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_DIRICHLET0 = 0, OR_BC_NOFLUX = 1 };
enum { OR_MEM_FULL = 0, OR_MEM_SHORT = 1, OR_MEM_ADAPTIVE = 2 };
enum { OR_ADAPT_PAPER = 0, OR_ADAPT_PARTITION = 1 };

typedef struct {
    int ndim;          /* 1, 2 or 3 */
    int nx, ny;        /* interior points per axis (ny = 1 in 1-D); point (x, y, z) at (z*ny + y)*nx + x */
    double gamma;      /* anomalous exponent */
    double alpha;      /* diffusivity */
    double dt, dx;     /* time step and grid spacing */
    int bc;            /* OR_BC_DIRICHLET0: zero ghosts; OR_BC_NOFLUX: mirror ghost (u_-1 = u_0) */
    double react[4];   /* f(u) = react[0] + react[1] u + react[2] u^2 + react[3] u^3 */
    int mem_mode;      /* OR_MEM_FULL | OR_MEM_SHORT | OR_MEM_ADAPTIVE */
    int mem_L;         /* short memory: lags 0..min(mem_L, k)  (eq. frac_shortmemory) */
    int mem_a;         /* adaptive memory: base interval [0, a], a >= 2 (Definition 3.1) */
    int adaptive_rule; /* OR_ADAPT_PAPER (literal Proposition 3.1) | OR_ADAPT_PARTITION */
    int nz;            /* points along the third axis (3-D; 1 otherwise) */
} or_problem;

/* Grunwald-Letnikov weights psi(g, m), m = 0..n-1, by the recurrence of
 * Section 2.1: psi(g,0) = 1, psi(g,m) = -psi(g,m-1) (2-g-m)/m.  If dpsi is not
 * NULL it receives d psi / d g by differentiating the same recurrence. */
int or_weights(double gamma, long n, double *psi, double *dpsi);

/* Memory terms used at step k, in ascending lag order: lag[t] and integer
 * multiplicity mult[t] (the increment length d = 2i-1 for a sampled median,
 * 1 otherwise).  Arrays must hold k+1 entries.  Returns the term count, or
 * -1 on bad arguments.  Full: eq. frac_final; short: eq. frac_shortmemory;
 * adaptive: Definitions 3.1, 3.2 and Proposition 3.1 (eq. eq:adapttime). */
long or_schedule(int mem_mode, long L, long a, int rule, long k, long *lag, long *mult);

/* Forward run of K steps from u0 (N = nx*ny doubles).  uK receives u^K.
 * If tape is not NULL it receives u^0..u^K ((K+1)*N doubles).
 * threads <= 0 uses the OpenMP default.  Returns 0, or -1 on bad arguments,
 * -2 on allocation failure. */
int or_run(const or_problem *p, const double *u0, long K, double *uK, double *tape, int threads);

/* BF16 storage of a value: round to 8 significant bits, to nearest, ties to even (the 16-bit
 * brain floating-point format has FP32's exponent range and 8 significant bits). */
double or_round_bf16(double x);

/* or_run with history rows stored in BF16 beyond an FP32 window: at step k the lags
 * m <= head + (blk > 0 ? k mod blk : 0) use delta^{k-m} as computed, older lags its BF16
 * rounding.  This is the storage rule of the mixed-precision GPU runs (not part of the paper):
 * per-step kernel blk = 0, head = its FP32 head lags; blocked kernel blk = head = the block
 * length.  With head >= K it equals or_run bit for bit. */
int or_run_bf16(const or_problem *p, const double *u0, long K, long blk, long head, double *uK, int threads);

/* Closed-loop adaptive memory (a reading of the Discussion, Section 4: the spacing of the
 * backward sum follows the derivative of the past history, a form of feedback).  Each step starts
 * from the adaptive schedule of p (Definitions 3.1/3.2, Proposition 3.1).  A median m that stands
 * for an increment of d = 2i-1 lags m-i+1 .. m+i-1 is kept, with weight d psi_m, only while the
 * history is smooth across the increment:
 *     V = (sum over the increment's rows r but its oldest of D_r) / M_{k-m}  <  tau,
 * where D_r = max_j |delta^r_j - delta^{r-1}_j| and M_r = max_j |delta^r_j| are computed once per
 * row (V bounds the relative change of the history across the increment, field-wide so that
 * every point shares one schedule; tau = +inf keeps every median).  Otherwise the increment's lags are summed one by one with
 * weight psi.  tau = +inf gives or_run's adaptive result bit for bit; tau = 0 with the partition
 * rule gives full memory.  *nterms (if not NULL) receives the number of (lag, weight) terms used
 * over the run, lag 0 included.  *margin (if not NULL) receives the smallest |V - tau| / tau over
 * the decisions with M_{k-m} > 0 (+inf for tau = +inf or 0, or without such decisions): how far
 * every decision lies from flipping, for comparisons with runs whose delta differs by rounding.
 * Returns as or_run. */
int or_run_closed(const or_problem *p, const double *u0, long K, double tau, double *uK, long *nterms,
                  double *margin, int threads);

/* Forward run in double complex (complex-step differentiation): the
 * imaginary parts of u0, gamma, alpha and react carry the perturbation.
 * Plain (uncompensated) summation.  Returns u^K as separate re/im arrays. */
int or_run_cs(const or_problem *p, double gamma_im, double alpha_im, const double react_im[4],
              const double *u0_re, const double *u0_im, long K, double *uK_re, double *uK_im);

/* FP64 reverse-time adjoint of the scheme for J = 1/2 sum_j (u^K_j - target_j)^2, following
 * the discrete Lagrangian of eq. frac_final:  lambda^K = u^K - target,
 *   g^r  = sum_{m=0}^{K-1-r} w_{r+m}(m) psi_m  lambda^{r+1+m},
 *   g'^r = sum_{m=0}^{K-1-r} w_{r+m}(m) psi'_m lambda^{r+1+m},
 *   lambda^r = lambda^{r+1} + dt f'(u^r) lambda^{r+1} + S L^T g^r,
 * where w_k(m) is the multiplicity of lag m in step k's schedule: delta^r enters step k = r+m
 * with weight w_k(m) psi_m.  Full memory: w = 1.  Short memory: w = 1 for m <= L, else 0
 * (eq. frac_shortmemory).  Adaptive memory: w_k(m) read from or_schedule(k) for every k
 * (Definitions 3.1/3.2, Proposition 3.1; d at a median, 1 on the base interval and the tail).
 * S = alpha dt^g / dx^2, dJ/dalpha = (S/alpha) sum_r <L u^r, g^r>,
 * dJ/dgamma = S sum_r (ln dt <L u^r, g^r> + <L u^r, g'^r>),
 * dJ/dreact_i = dt sum_r <lambda^{r+1}, (u^r)^i>, dJ/du0 = lambda^0.
 * Adaptive memory keeps a K x K table of multiplicities.  Any output pointer may be NULL. */
int or_adjoint(const or_problem *p, const double *u0, long K, const double *target,
               double *J, double *dJ_du0, double *dJ_dgamma, double *dJ_dalpha,
               double dJ_dreact[4], int threads);

/* Scalar recursion of one Laplacian eigenmode (L phi = -Lambda phi) under
 * the scheme with linear reaction f(u) = r1 u:
 *   A^{k+1} = A^k + dt r1 A^k - S Lambda sum_{(m,d) in sched(k)} d psi_m A^{k-m}.
 * out receives A^0..A^K (K+1 doubles). */
int or_scalar_mode(double gamma, double alpha, double dt, double dx, double r1, double Lambda,
                   int mem_mode, long L, long a, int rule, double A0, long K, double *out);

#ifdef __cplusplus
}
#endif
#endif

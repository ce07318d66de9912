/*
 * FP64 CPU oracle of GATE's TE iteration -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, plain reference that the CUDA path is checked
 * against.  Only the test suite, the package's smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library; both sides only read the same generated instance.
 *
 * What it computes (GATE, Section 3):
 *   maximise  sum_c U_alpha(S_c),  S_c = sum_{r in P_c} x_r           (Eq. 4)
 *   s.t.      S_c <= D_c (Eq. 1),  sum_{r ni e} x_r <= C_e (Eq. 2),  x >= 0 (Eq. 3)
 * by ADMM on the consensus reformulation x_r = y_{e,r} (Eqs. 5-6) of the
 * augmented Lagrangian (Eq. 7), read as the standard two-block scaled ADMM
 * that the convergence proof (Appendix C, Part I) invokes:
 *   x-block : one subproblem per demand holding the utility, the demand cap
 *             and non-negativity (Section 3.3 "Rate Updates", Appendix B.2);
 *   y-block : one subproblem per edge, the projection onto sum_r y_{e,r} <= C_e
 *             (Section 3.3 "Rate Suggestion Updates");
 *   dual    : the scaled consensus duals u_{e,r} (Eq. 10).
 * Starting from u = 0 (Algorithm 1, initialisation) the consensus dual of an
 * edge is the same for every path on it, so the oracle stores one scaled price
 * u_e per edge and the per-incidence primal residual d_e = x_r - y_{e,r}
 * (also one value per edge).  The function or_run_expanded keeps every
 * y_{e,r} and u_{e,r} explicitly; the tests check that both agree.
 *
 * Per iteration (Algorithm 1, in ADMM order x -> y -> u):
 *   m_r  = x_r - (1/n_r) sum_{e in r} (u_e + d_e)        consensus target
 *   x_r' = max(0, m_r + lambda_c / (beta n_r))           per-demand split, with
 *          lambda_c = min(lambda*, lambda_D): lambda* from the sum equation
 *          S = sum_r max(0, m_r + S^-alpha/(beta n_r)) (Appendix B.2,
 *          Newton-bisection), lambda_D from S(lambda) = D_c (demand cap)
 *   L_e  = sum_{r ni e} x_r'                              edge loads
 *   u_e' = max(0, u_e + (L_e - C_e)/n_e),  d_e' = u_e' - u_e   (Eq. 9 / Eq. 13
 *          after the collapse; n_e = number of paths on e)
 *   s    = ||x' - x|| / ||x'||                           dual residual (Eq. 15)
 *   r    = sqrt(sum_e n_e d_e'^2) / sqrt(sum_r n_r x_r'^2)   primal residual (Eq. 16)
 *   beta : residual balancing (Eq. 17) while max(r, s) exceeds a floor
 *          (default 1e-6, the rounding level of the FP32 iteration), beta
 *          kept within [1e-30, 1e30]; on a change the scaled duals u are
 *          multiplied by beta_old/beta_new and d (a primal quantity) is kept
 *   stop : r <= gamma and s <= gamma (Eq. 18) with alpha-continuation
 *          (Section 3.4 "alpha-increments", Algorithm 1); optionally also
 *          the primal residual in the max norm, the largest relative
 *          capacity violation max_e n_e |u_e' - u_e| / C_e <= gamma_max
 * Values are normalised by scale = max_e C_e (the alpha-fair argmax is
 * invariant to a common scaling of C and D).
 *
 * Also here: the feasibility projection (Algorithm 2), a proportional
 * feasibility scaling (not in the paper) and the duality gap of a feasible
 * allocation.  Parallel loops (OpenMP) run over independent
 * demands or edges only, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n_edges;
    int32_t n_demands;
    int64_t n_paths;
    int64_t nnz;
    const double* cap;      /* [E]   capacities C_e                       */
    const double* demand;   /* [K]   demands D_c                          */
    const int64_t* dpo;     /* [K+1] demand -> path offsets               */
    const int64_t* peo;     /* [P+1] path -> incidence offsets            */
    const int32_t* pe;      /* [nnz] edge ids                             */
} or_instance;

typedef struct {
    double alpha_target;  /* INFINITY: max-min fairness                   */
    double alpha_start;   /* first alpha of the continuation (0)          */
    double alpha_step;    /* continuation increment (1)                   */
    double alpha_max;     /* continuation cap                             */
    double gamma;         /* convergence threshold (1e-3)                 */
    double gamma_max;     /* > 0: convergence also needs max_e n_e |du_e| / C_e <= gamma_max */
    double A, C;          /* residual balancing constants (10, 2)         */
    double beta0;         /* initial penalty, normalised units (1)        */
    double beta_max;      /* > 0: balancing never raises beta above beta_max * beta0 */
    double balance_floor; /* residual balancing only while max(r, s) exceeds it */
    int32_t adapt_beta;   /* 1: residual balancing on                     */
    int32_t continuation; /* 1: stop when converged on the first iteration after an increment */
    int32_t threads;      /* OpenMP threads (0: runtime default)          */
    int32_t scale_mode;   /* unit of the normalised problem: 0 = max_e C_e, 2 = 1 (caller units),
                             1 = geometric mean of the demands            */
} or_options;

/* Scalars of the solver state (arrays are passed separately). */
typedef struct {
    double beta, alpha, scale;
    double beta0;        /* initial penalty                               */
    int64_t iter;        /* iterations run so far                        */
    int64_t iter_alpha;  /* iterations since alpha last changed          */
    int32_t converged;   /* 1 once the stop rule fired                   */
    int32_t pad;
} or_scalars;

enum { TR_R = 0, TR_S, TR_BETA, TR_ALPHA, TR_EVENT, TR_WIDTH };

/* Field-by-field copy of the option and scalar structs into doubles, so the
 * tests can check the ctypes mirrors against this file's layout. */
void or_echo_options(const or_options* o, double* out) {
    out[0] = o->alpha_target; out[1] = o->alpha_start; out[2] = o->alpha_step; out[3] = o->alpha_max;
    out[4] = o->gamma; out[5] = o->gamma_max; out[6] = o->A; out[7] = o->C; out[8] = o->beta0;
    out[9] = o->beta_max; out[10] = o->balance_floor; out[11] = o->adapt_beta; out[12] = o->continuation;
    out[13] = o->threads; out[14] = o->scale_mode; out[15] = (double)sizeof(or_options);
}
void or_echo_scalars(const or_scalars* sc, double* out) {
    out[0] = sc->beta; out[1] = sc->alpha; out[2] = sc->scale; out[3] = sc->beta0; out[4] = (double)sc->iter;
    out[5] = (double)sc->iter_alpha; out[6] = sc->converged; out[7] = (double)sizeof(or_scalars);
}

/* ------------------------------------------------------------------ */
/* alpha-fair utility, Eq. 4                                           */
/* ------------------------------------------------------------------ */
double or_utility(double S, double alpha) {
    if (alpha == 1.0) return log(S);
    return (pow(S, 1.0 - alpha) - 1.0) / (1.0 - alpha);
}

/* ------------------------------------------------------------------ */
/* Per-demand x-block (Section 3.3 "Rate Updates", Appendix B.2).      */
/*                                                                      */
/* minimise -U_alpha(S) + sum_r (1/(2 w_r)) (x_r - m_r)^2                */
/*   s.t. x >= 0, S = sum_r x_r <= D,   with w_r = 1/(beta n_r).         */
/* Stationarity gives x_r = max(0, m_r + lambda w_r) with lambda =       */
/* U'(S) - mu, mu >= 0 the demand-cap multiplier.  Writes x_out and      */
/* returns lambda.                                                       */
/* ------------------------------------------------------------------ */
/* G(S) = sum_r max(0, m_r + w_r S^-alpha): the sum implied by a candidate
 * total S when the demand cap is slack (lambda = S^-alpha). */
static double G_of_S(int n, const double* m, const double* w, double S, double alpha, double* dG) {
    double lam = exp(-alpha * log(S));
    double G = 0.0, H = 0.0;
    for (int i = 0; i < n; ++i) {
        double v = m[i] + lam * w[i];
        if (v > 0.0) { G += v; H += w[i]; }
    }
    /* d lambda / dS = -alpha S^(-alpha-1) */
    if (dG) *dG = H * (-alpha * lam / S);
    return G;
}

double or_demand_solve(int n, const double* m, const double* w, double D, double alpha, double* x_out) {
    /* sort paths by breakpoint b_r = -m_r / w_r (path r active for lambda > b_r) */
    int idx_small[64];
    int* idx = n <= 64 ? idx_small : (int*)malloc(sizeof(int) * (size_t)n);
    double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) { idx[i] = i; b[i] = -m[i] / w[i]; }
    for (int i = 1; i < n; ++i) {               /* insertion sort, stable */
        int v = idx[i];
        int j = i - 1;
        while (j >= 0 && b[idx[j]] > b[v]) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = v;
    }
    /* lambda_D: S(lambda) = D.  S is piecewise linear and increasing; on the
     * segment after the j-th breakpoint the active paths are the first j in
     * breakpoint order, S = A_j + H_j lambda. */
    double A = 0.0, H = 0.0, lamD = 0.0;
    int found = 0;
    for (int j = 0; j < n && !found; ++j) {
        const double bj = b[idx[j]];
        if (j > 0 && A + H * bj >= D) {           /* S at this breakpoint already >= D */
            lamD = (D - A) / H;
            found = 1;
            break;
        }
        A += m[idx[j]];
        H += w[idx[j]];
    }
    if (!found) lamD = (D - A) / H;
    double lam;
    if (alpha == 0.0) {
        /* U' = 1: lambda = min(1, lambda_D) */
        lam = lamD < 1.0 ? lamD : 1.0;
    } else if (lamD <= 0.0 || log(lamD) + alpha * log(D) <= 0.0) {
        /* lambda_D <= U'(D): the demand cap binds */
        lam = lamD;
    } else {
        /* cap slack: solve F(S) = S - G(S) = 0 on (0, D) by Newton-bisection
         * (Appendix B.2).  F(0+) < 0 < F(D), F increasing. */
        double lo = 0.0, hi = D, S = D;
        double dG;
        for (int it = 0; it < 400; ++it) {
            double G = G_of_S(n, m, w, S, alpha, &dG);
            double F = S - G;
            if (F > 0.0) hi = S; else lo = S;
            if (F == 0.0) break;
            double dF = 1.0 - dG;                   /* > 0 */
            double Sn = S - F / dF;
            if (!(Sn > lo && Sn < hi)) Sn = 0.5 * (lo + hi);
            if (fabs(Sn - S) <= 1e-15 * S || hi - lo <= 1e-15 * hi) { S = Sn; break; }
            S = Sn;
        }
        lam = exp(-alpha * log(S));
        if (lam > lamD) lam = lamD;
    }
    for (int i = 0; i < n; ++i) {
        double v = m[i] + lam * w[i];
        x_out[i] = v > 0.0 ? v : 0.0;
    }
    free(b);
    if (idx != idx_small) free(idx);
    return lam;
}

/* ------------------------------------------------------------------ */
/* Edge -> path incidence (CSC) for the loads L_e = sum_{r ni e} x_r.   */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t* off;   /* [E+1] */
    int64_t* path;  /* [nnz] path ids, ascending per edge */
} or_csc;

static void csc_build(const or_instance* I, or_csc* T) {
    const int E = I->n_edges;
    T->off = (int64_t*)calloc((size_t)E + 1, sizeof(int64_t));
    T->path = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I->nnz > 0 ? I->nnz : 1));
    for (int64_t i = 0; i < I->nnz; ++i) T->off[I->pe[i] + 1]++;
    for (int e = 0; e < E; ++e) T->off[e + 1] += T->off[e];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    memcpy(fill, T->off, sizeof(int64_t) * (size_t)E);
    for (int64_t r = 0; r < I->n_paths; ++r)
        for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) T->path[fill[I->pe[i]]++] = r;
    free(fill);
}

static void csc_free(or_csc* T) { free(T->off); free(T->path); }

static int64_t max_paths_per_demand(const or_instance* I) {
    int64_t mx = 0;
    for (int32_t c = 0; c < I->n_demands; ++c) {
        int64_t k = I->dpo[c + 1] - I->dpo[c];
        if (k > mx) mx = k;
    }
    return mx;
}

/* ------------------------------------------------------------------ */
/* Initial state (Algorithm 1): x^0 = D_c/|P_c| unless x0 is given,     */
/* duals zero.  Arrays x[P], u[E], d[E] are normalised by scale.        */
/* ------------------------------------------------------------------ */
int or_init(const or_instance* I, const or_options* o, const double* x0, double* x, double* u,
            double* d, or_scalars* sc) {
    double scale = 0.0;
    if (o->scale_mode == 1) {
        double lg = 0.0;
        for (int32_t c = 0; c < I->n_demands; ++c) lg += log(I->demand[c]);
        scale = exp(lg / (double)I->n_demands);
    } else if (o->scale_mode == 2) {
        scale = 1.0;  /* caller units */
    } else {
        for (int e = 0; e < I->n_edges; ++e) if (I->cap[e] > scale) scale = I->cap[e];
    }
    if (!(scale > 0.0)) return 1;
    for (int32_t c = 0; c < I->n_demands; ++c) {
        const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
        for (int64_t r = p0; r < p1; ++r)
            x[r] = x0 ? x0[r] / scale : (I->demand[c] / scale) / (double)(p1 - p0);
    }
    for (int e = 0; e < I->n_edges; ++e) { u[e] = 0.0; d[e] = 0.0; }
    if (o->beta0 > 0.0) {
        sc->beta = o->beta0;
    } else {
        /* beta0 <= 0: the first push lambda/(beta n_r) at lambda = 1 equals
         * the mean initial path rate: beta0 = 1 / (mean n_r * mean x^0_r) */
        double xs = 0.0;
        for (int64_t r = 0; r < I->n_paths; ++r) xs += x[r];
        const double xbar = xs / (double)I->n_paths;
        const double nbar = (double)I->nnz / (double)I->n_paths;
        sc->beta = 1.0 / (nbar * xbar);
    }
    sc->beta0 = sc->beta;
    sc->alpha = isfinite(o->alpha_target) && o->alpha_start > o->alpha_target ? o->alpha_target : o->alpha_start;
    sc->scale = scale;
    sc->iter = 0;
    sc->iter_alpha = 0;
    sc->converged = 0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Run up to max_iters iterations (stops early on convergence).         */
/* trace (optional): TR_WIDTH doubles per iteration.                    */
/* Returns the number of iterations run in this call.                   */
/* ------------------------------------------------------------------ */
int64_t or_run(const or_instance* I, const or_options* o, double* x, double* u, double* d,
               or_scalars* sc, int64_t max_iters, double* trace) {
#ifdef _OPENMP
    if (o->threads > 0) omp_set_num_threads(o->threads);
#endif
    const int E = I->n_edges;
    const int64_t P = I->n_paths;
    const double scale = sc->scale;
    double* C = (double*)malloc(sizeof(double) * (size_t)E);
    double* D = (double*)malloc(sizeof(double) * (size_t)(I->n_demands > 0 ? I->n_demands : 1));
    int64_t* ne = (int64_t*)calloc((size_t)E, sizeof(int64_t));
    for (int e = 0; e < E; ++e) C[e] = I->cap[e] / scale;
    for (int32_t c = 0; c < I->n_demands; ++c) D[c] = I->demand[c] / scale;
    for (int64_t i = 0; i < I->nnz; ++i) ne[I->pe[i]]++;
    or_csc T;
    csc_build(I, &T);
    double* xn = (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
    double* L = (double*)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double* un = (double*)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    const int64_t kmax = max_paths_per_demand(I);

    int64_t done = 0;
    while (done < max_iters && !sc->converged) {
        const double beta = sc->beta, alpha = sc->alpha;
        /* x-block: one subproblem per demand */
#ifdef _OPENMP
#pragma omp parallel
#endif
        {
            double* m = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
            double* w = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int32_t c = 0; c < I->n_demands; ++c) {
                const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
                const int n = (int)(p1 - p0);
                for (int j = 0; j < n; ++j) {
                    const int64_t r = p0 + j;
                    const int64_t nr = I->peo[r + 1] - I->peo[r];
                    double q = 0.0;
                    for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) q += u[I->pe[i]] + d[I->pe[i]];
                    m[j] = x[r] - q / (double)nr;
                    w[j] = 1.0 / (beta * (double)nr);
                }
                or_demand_solve(n, m, w, D[c], alpha, xn + p0);
            }
            free(m);
            free(w);
        }
        /* y-block + dual: loads, then the per-edge price */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int e = 0; e < E; ++e) {
            double s = 0.0;
            for (int64_t i = T.off[e]; i < T.off[e + 1]; ++i) s += xn[T.path[i]];
            L[e] = s;
            un[e] = ne[e] > 0 ? fmax(0.0, u[e] + (s - C[e]) / (double)ne[e]) : 0.0;
        }
        /* residuals (sequential sums, fixed order) */
        double ds2 = 0.0, x2 = 0.0, ex2 = 0.0, r2 = 0.0, rmax = 0.0;
        for (int64_t r = 0; r < P; ++r) {
            const double dx = xn[r] - x[r];
            const double nr = (double)(I->peo[r + 1] - I->peo[r]);
            ds2 += dx * dx;
            x2 += xn[r] * xn[r];
            ex2 += nr * xn[r] * xn[r];
        }
        for (int e = 0; e < E; ++e) {
            const double de = un[e] - u[e];
            r2 += (double)ne[e] * de * de;
            if (ne[e] > 0) rmax = fmax(rmax, (double)ne[e] * fabs(de) / C[e]);
            d[e] = de;
            u[e] = un[e];
        }
        memcpy(x, xn, sizeof(double) * (size_t)P);
        const double s_res = sqrt(ds2) / fmax(sqrt(x2), 1e-30);
        const double r_res = sqrt(r2) / fmax(sqrt(ex2), 1e-30);
        sc->iter++;
        sc->iter_alpha++;
        done++;
        int event = 0;
        /* residual balancing, Eq. 17, while the residuals are above the
         * floor (below it they are rounding noise of the FP32 iteration, so
         * both sides skip the step), keeping beta within [1e-30, 1e30] */
        if (o->adapt_beta && fmax(r_res, s_res) > o->balance_floor) {
            double nb = beta;
            if (r_res > o->A * s_res) nb = beta * o->C;
            else if (s_res > o->A * r_res) nb = beta / o->C;
            if (!(nb >= 1e-30 && nb <= 1e30)) nb = beta;
            if (o->beta_max > 0.0 && nb > o->beta_max * sc->beta0) nb = beta;
            if (nb != beta) {
                const double ratio = beta / nb;
                for (int e = 0; e < E; ++e) u[e] *= ratio;
                sc->beta = nb;
                event |= 1;
            }
        }
        /* convergence and alpha-continuation, Eq. 18 and Algorithm 1 */
        if (r_res <= o->gamma && s_res <= o->gamma && (o->gamma_max <= 0.0 || rmax <= o->gamma_max)) {
            if (sc->alpha >= o->alpha_target) {
                sc->converged = 1;
                event |= 4;
            } else if (o->continuation && sc->iter_alpha == 1 && sc->alpha > o->alpha_start) {
                sc->converged = 1;
                event |= 8;
            } else if (sc->alpha >= o->alpha_max) {
                sc->converged = 1;
                event |= 16;
            } else {
                double na = sc->alpha + o->alpha_step;
                if (na > o->alpha_target) na = o->alpha_target;
                if (na > o->alpha_max) na = o->alpha_max;
                sc->alpha = na;
                sc->iter_alpha = 0;
                event |= 2;
            }
        }
        if (trace) {
            double* t = trace + (done - 1) * TR_WIDTH;
            t[TR_R] = r_res;
            t[TR_S] = s_res;
            t[TR_BETA] = sc->beta;
            t[TR_ALPHA] = sc->alpha;
            t[TR_EVENT] = (double)event;
        }
    }
    free(C); free(D); free(ne); free(xn); free(L); free(un);
    csc_free(&T);
    return done;
}

/* ------------------------------------------------------------------ */
/* The same iteration with every consensus copy y_{e,r} and scaled dual  */
/* u_{e,r} stored per incidence (Eqs. 5-7, 10, 13 as two-block ADMM),    */
/* fixed beta and alpha, single-threaded.  Used only to check the        */
/* per-edge collapse above.  x[P] in/out (normalised), y[nnz], u[nnz]    */
/* in/out; y starts at x and u at 0.                                     */
/* ------------------------------------------------------------------ */
void or_run_expanded(const or_instance* I, double beta, double alpha, double scale, double* x,
                     double* y, double* uu, int64_t iters) {
    const int E = I->n_edges;
    const int64_t P = I->n_paths;
    const int64_t kmax = max_paths_per_demand(I);
    double* m = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
    double* V = (double*)calloc((size_t)E, sizeof(double));
    int64_t* ne = (int64_t*)calloc((size_t)E, sizeof(int64_t));
    for (int64_t i = 0; i < I->nnz; ++i) ne[I->pe[i]]++;
    for (int64_t k = 0; k < iters; ++k) {
        /* x-block: argmin -U + (beta/2) sum_{e in r} (x_r - y_{e,r} + u_{e,r})^2 */
        for (int32_t c = 0; c < I->n_demands; ++c) {
            const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
            const int n = (int)(p1 - p0);
            for (int j = 0; j < n; ++j) {
                const int64_t r = p0 + j;
                const int64_t nr = I->peo[r + 1] - I->peo[r];
                double acc = 0.0;
                for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) acc += y[i] - uu[i];
                m[j] = acc / (double)nr;
                w[j] = 1.0 / (beta * (double)nr);
            }
            or_demand_solve(n, m, w, I->demand[c] / scale, alpha, x + p0);
        }
        /* y-block: per edge, project v_{e,r} = x_r + u_{e,r} onto sum_r y <= C_e */
        for (int e = 0; e < E; ++e) V[e] = 0.0;
        for (int64_t r = 0; r < P; ++r)
            for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) V[I->pe[i]] += x[r] + uu[i];
        for (int e = 0; e < E; ++e)
            V[e] = ne[e] > 0 ? fmax(0.0, (V[e] - I->cap[e] / scale) / (double)ne[e]) : 0.0;
        for (int64_t r = 0; r < P; ++r)
            for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) {
                y[i] = x[r] + uu[i] - V[I->pe[i]];
                /* dual: u += x - y */
                uu[i] += x[r] - y[i];
            }
    }
    free(m); free(w); free(V); free(ne);
}

/* ------------------------------------------------------------------ */
/* Gradient of the fairness objective through K iterations (not in the  */
/* paper; the differentiated form for capacity planning).               */
/*                                                                      */
/* J(C, D) = sum_c U_alpha(scale S_c^K), S_c^K the demand totals of the */
/* iterate after K iterations from the initial state of Algorithm 1, with */
/* beta and alpha fixed (no residual balancing, no continuation) and the */
/* normalisation unit scale held fixed.  gC[e] = dJ/dC_e, gD[c] = dJ/dD_c */
/* (caller units), by reverse-mode differentiation of every step:       */
/*   x-block: on the active set A of a demand (x' > 0), x' = m + lambda w */
/*     with w = 1/(beta n_r); if the demand cap binds (lambda below       */
/*     U'(S)), lambda = (D - sum_A m) / sum_A w; else lambda = U'(S) and   */
/*     d lambda = -alpha lambda / (S + alpha lambda sum_A w) d(sum_A m)    */
/*   u' = max(0, u + (L - C)/n_e), d' = u' - u, L = sum of x' over e      */
/*   m = x - (1/n_r) sum_{e in r} (u_e + d_e)                             */
/* States are kept every ckpt iterations and each segment is recomputed  */
/* forward before its reverse sweep.  Returns 0, or 1 on bad options.    */
/* ------------------------------------------------------------------ */
static double utility_d(double S, double alpha) { return alpha == 0.0 ? 1.0 : exp(-alpha * log(S)); }

/* one forward iteration with fixed beta, alpha: (x, u, d) -> next, in place */
static void fwd_step(const or_instance* I, const double* Cn, const double* Dn, const int64_t* ne, const or_csc* T,
                     double beta, double alpha, double* x, double* u, double* d, double* xn, double* m, double* w) {
    for (int32_t c = 0; c < I->n_demands; ++c) {
        const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
        const int n = (int)(p1 - p0);
        for (int j = 0; j < n; ++j) {
            const int64_t r = p0 + j;
            const int64_t nr = I->peo[r + 1] - I->peo[r];
            double q = 0.0;
            for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) q += u[I->pe[i]] + d[I->pe[i]];
            m[j] = x[r] - q / (double)nr;
            w[j] = 1.0 / (beta * (double)nr);
        }
        or_demand_solve(n, m, w, Dn[c], alpha, xn + p0);
    }
    for (int e = 0; e < I->n_edges; ++e) {
        double L = 0.0;
        for (int64_t i = T->off[e]; i < T->off[e + 1]; ++i) L += xn[T->path[i]];
        const double un = ne[e] > 0 ? fmax(0.0, u[e] + (L - Cn[e]) / (double)ne[e]) : 0.0;
        d[e] = un - u[e];
        u[e] = un;
    }
    memcpy(x, xn, sizeof(double) * (size_t)I->n_paths);
}

int or_gradient(const or_instance* I, const or_options* o, int64_t K, int64_t ckpt, double* J, double* gC,
                double* gD) {
    if (K < 0 || ckpt < 1 || !(o->beta0 > 0.0) || o->adapt_beta || o->continuation) return 1;
    const int E = I->n_edges;
    const int32_t NC = I->n_demands;
    const int64_t P = I->n_paths;
    or_scalars sc;
    double* x = (double*)malloc(sizeof(double) * (size_t)P);
    double* u = (double*)malloc(sizeof(double) * (size_t)E);
    double* d = (double*)malloc(sizeof(double) * (size_t)E);
    if (or_init(I, o, NULL, x, u, d, &sc)) { free(x); free(u); free(d); return 1; }
    const double scale = sc.scale, beta = sc.beta, alpha = sc.alpha;
    double* Cn = (double*)malloc(sizeof(double) * (size_t)E);
    double* Dn = (double*)malloc(sizeof(double) * (size_t)NC);
    int64_t* ne = (int64_t*)calloc((size_t)E, sizeof(int64_t));
    for (int e = 0; e < E; ++e) Cn[e] = I->cap[e] / scale;
    for (int32_t c = 0; c < NC; ++c) Dn[c] = I->demand[c] / scale;
    for (int64_t i = 0; i < I->nnz; ++i) ne[I->pe[i]]++;
    or_csc T;
    csc_build(I, &T);
    const int64_t kmax = max_paths_per_demand(I);
    double* m = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
    double* xs = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
    double* xn = (double*)malloc(sizeof(double) * (size_t)P);
    /* forward with checkpoints at k = 0, ckpt, 2 ckpt, ... */
    const int64_t nck = K / ckpt + 1;
    double* ck = (double*)malloc(sizeof(double) * (size_t)nck * (size_t)(P + 2 * E));
    for (int64_t k = 0; k < K; ++k) {
        if (k % ckpt == 0) {
            double* c0 = ck + (size_t)(k / ckpt) * (size_t)(P + 2 * E);
            memcpy(c0, x, sizeof(double) * (size_t)P);
            memcpy(c0 + P, u, sizeof(double) * (size_t)E);
            memcpy(c0 + P + E, d, sizeof(double) * (size_t)E);
        }
        fwd_step(I, Cn, Dn, ne, &T, beta, alpha, x, u, d, xn, m, w);
    }
    /* objective and its adjoint at x^K */
    double* xb = (double*)calloc((size_t)P, sizeof(double));
    double* ub = (double*)calloc((size_t)E, sizeof(double));
    double* db = (double*)calloc((size_t)E, sizeof(double));
    double* Cb = (double*)calloc((size_t)E, sizeof(double));
    double* Db = (double*)calloc((size_t)NC, sizeof(double));
    double Jv = 0.0;
    for (int32_t c = 0; c < NC; ++c) {
        double S = 0.0;
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) S += x[r];
        Jv += or_utility(scale * S, alpha);
        const double g = scale * utility_d(scale * S, alpha);  /* dJ/dS_c */
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) xb[r] = g;
    }
    /* reverse sweep, one checkpoint segment at a time */
    const int64_t seg = ckpt;
    double* sx = (double*)malloc(sizeof(double) * (size_t)(seg + 1) * (size_t)P);
    double* su = (double*)malloc(sizeof(double) * (size_t)(seg + 1) * (size_t)E);
    double* sd = (double*)malloc(sizeof(double) * (size_t)(seg + 1) * (size_t)E);
    double* Lb = (double*)malloc(sizeof(double) * (size_t)E);
    double* gb = (double*)malloc(sizeof(double) * (size_t)P);
    double* qb = (double*)malloc(sizeof(double) * (size_t)P);
    for (int64_t k0 = ((K - 1) / ckpt) * ckpt; K > 0 && k0 >= 0; k0 -= ckpt) {
        const int64_t k1 = (k0 + ckpt < K) ? k0 + ckpt : K;
        const double* c0 = ck + (size_t)(k0 / ckpt) * (size_t)(P + 2 * E);
        memcpy(x, c0, sizeof(double) * (size_t)P);
        memcpy(u, c0 + P, sizeof(double) * (size_t)E);
        memcpy(d, c0 + P + E, sizeof(double) * (size_t)E);
        for (int64_t k = k0; k <= k1; ++k) {
            memcpy(sx + (size_t)(k - k0) * P, x, sizeof(double) * (size_t)P);
            memcpy(su + (size_t)(k - k0) * E, u, sizeof(double) * (size_t)E);
            memcpy(sd + (size_t)(k - k0) * E, d, sizeof(double) * (size_t)E);
            if (k < k1) fwd_step(I, Cn, Dn, ne, &T, beta, alpha, x, u, d, xn, m, w);
        }
        for (int64_t k = k1 - 1; k >= k0; --k) {
            const double* xk = sx + (size_t)(k - k0) * P;
            const double* uk = su + (size_t)(k - k0) * E;
            const double* dk = sd + (size_t)(k - k0) * E;
            const double* u1 = su + (size_t)(k + 1 - k0) * E;
            /* d' = u' - u and u' = max(0, u + (L - C)/n_e) */
            for (int e = 0; e < E; ++e) {
                const double tot = ub[e] + db[e];
                double uin = -db[e];
                Lb[e] = 0.0;
                if (ne[e] > 0 && u1[e] > 0.0) {
                    uin += tot;
                    Lb[e] = tot / (double)ne[e];
                    Cb[e] -= tot / (double)ne[e];
                }
                ub[e] = uin;
                db[e] = 0.0;
            }
            /* L = sum of x' over each edge */
            for (int64_t r = 0; r < P; ++r) {
                double g = xb[r];
                for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) g += Lb[I->pe[i]];
                gb[r] = g;
            }
            /* x-block of each demand */
            for (int32_t c = 0; c < NC; ++c) {
                const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
                const int n = (int)(p1 - p0);
                for (int j = 0; j < n; ++j) {
                    const int64_t r = p0 + j;
                    const int64_t nr = I->peo[r + 1] - I->peo[r];
                    double q = 0.0;
                    for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) q += uk[I->pe[i]] + dk[I->pe[i]];
                    m[j] = xk[r] - q / (double)nr;
                    w[j] = 1.0 / (beta * (double)nr);
                }
                const double lam = or_demand_solve(n, m, w, Dn[c], alpha, xs);
                double S = 0.0, WA = 0.0, G = 0.0;
                for (int j = 0; j < n; ++j)
                    if (xs[j] > 0.0) {
                        S += xs[j];
                        WA += w[j];
                        G += gb[p0 + j] * w[j];
                    }
                double dl_dm = 0.0;  /* d lambda / d m_s for s in A */
                if (WA > 0.0) {
                    const int capped = lam < utility_d(S, alpha) * (1.0 - 1e-9);
                    if (capped) {
                        dl_dm = -1.0 / WA;
                        Db[c] += G / WA;
                    } else {
                        dl_dm = -alpha * lam / (S + alpha * lam * WA);
                    }
                }
                for (int j = 0; j < n; ++j) {
                    const int64_t r = p0 + j;
                    const double mb = xs[j] > 0.0 ? gb[r] + G * dl_dm : 0.0;
                    xb[r] = mb;  /* m = x - q/n_r */
                    qb[r] = -mb / (double)(I->peo[r + 1] - I->peo[r]);
                }
            }
            /* q = sum of (u + d) over the path's edges */
            for (int64_t r = 0; r < P; ++r)
                for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) {
                    ub[I->pe[i]] += qb[r];
                    db[I->pe[i]] += qb[r];
                }
        }
    }
    /* x^0 = D_c / |P_c| */
    for (int32_t c = 0; c < NC; ++c) {
        const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
        double s0 = 0.0;
        for (int64_t r = p0; r < p1; ++r) s0 += xb[r];
        Db[c] += s0 / (double)(p1 - p0);
    }
    for (int e = 0; e < E; ++e) gC[e] = Cb[e] / scale;
    for (int32_t c = 0; c < NC; ++c) gD[c] = Db[c] / scale;
    *J = Jv;
    free(x); free(u); free(d); free(Cn); free(Dn); free(ne); free(m); free(w); free(xs); free(xn); free(ck);
    free(xb); free(ub); free(db); free(Cb); free(Db); free(sx); free(su); free(sd); free(Lb); free(gb); free(qb);
    csc_free(&T);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Feasibility projection, Algorithm 2.  x[P] in/out (any units that    */
/* match cap and demand).  alpha is the fairness level of the score      */
/* score_p = S_c^alpha * C_p; ties go to the lower path index.  The edge */
/* step plans, for every violated edge independently from one snapshot   */
/* of x, the trims delta_p^e in descending score order; each path then  */
/* subtracts the largest trim planned for it over its edges.             */
/* ------------------------------------------------------------------ */
typedef struct { double key; int64_t path; } or_keyed;

static int keyed_cmp(const void* a, const void* b) {
    const or_keyed* p = (const or_keyed*)a;
    const or_keyed* q = (const or_keyed*)b;
    if (p->key > q->key) return -1;
    if (p->key < q->key) return 1;
    return (p->path < q->path) ? -1 : (p->path > q->path);
}

/* log of score_p = alpha log S_c + log C_p (-inf when the score is 0),
 * rounded to FP32: the order of Algorithm 2 is a decision taken on a
 * floating-point score, so it is taken in the CUDA path's precision (the
 * FP32 key of the FP64 score, S in caller units) and both sides order
 * near-equal scores alike */
static double log_score(double S, int64_t Cp, double alpha) {
    if (Cp <= 0) return -INFINITY;
    if (alpha == 0.0) return (double)(float)log((double)Cp);
    if (!(S > 0.0)) return -INFINITY;
    return (double)(float)(alpha * log(S) + log((double)Cp));
}

static void proj_aux(const or_instance* I, const double* x, double* S, double* L, int64_t* Cp) {
    for (int32_t c = 0; c < I->n_demands; ++c) {
        double s = 0.0;
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) s += x[r];
        S[c] = s;
    }
    for (int e = 0; e < I->n_edges; ++e) L[e] = 0.0;
    for (int64_t r = 0; r < I->n_paths; ++r)
        for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) L[I->pe[i]] += x[r];
    for (int64_t r = 0; r < I->n_paths; ++r) {
        int64_t cnt = 0;
        for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) cnt += (L[I->pe[i]] - I->cap[I->pe[i]] > 0.0);
        Cp[r] = cnt;
    }
}

void or_project(const or_instance* I, double* x, double alpha) {
    const int E = I->n_edges;
    const int64_t P = I->n_paths;
    double* S = (double*)malloc(sizeof(double) * (size_t)(I->n_demands > 0 ? I->n_demands : 1));
    double* L = (double*)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    int64_t* Cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    /* 1. non-negativity */
    for (int64_t r = 0; r < P; ++r) if (!(x[r] > 0.0)) x[r] = 0.0;
    /* 2. demand violations, greedy in descending score */
    proj_aux(I, x, S, L, Cp);
    const int64_t kmax = max_paths_per_demand(I);
    or_keyed* buf = (or_keyed*)malloc(sizeof(or_keyed) * (size_t)(kmax > 0 ? kmax : 1));
    for (int32_t c = 0; c < I->n_demands; ++c) {
        double Ec = S[c] - I->demand[c];
        if (!(Ec > 0.0)) continue;
        const int64_t p0 = I->dpo[c], p1 = I->dpo[c + 1];
        for (int64_t r = p0; r < p1; ++r) { buf[r - p0].key = log_score(S[c], Cp[r], alpha); buf[r - p0].path = r; }
        qsort(buf, (size_t)(p1 - p0), sizeof(or_keyed), keyed_cmp);
        for (int64_t j = 0; j < p1 - p0 && Ec > 0.0; ++j) {
            const int64_t r = buf[j].path;
            const double dx = fmin(Ec, x[r]);
            x[r] -= dx;
            Ec -= dx;
        }
    }
    free(buf);
    /* 3. recompute, then capacity violations (Jacobi plans, max per path) */
    proj_aux(I, x, S, L, Cp);
    or_csc T;
    csc_build(I, &T);
    double* trim = (double*)calloc((size_t)(P > 0 ? P : 1), sizeof(double));
    int64_t* pd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    for (int32_t c = 0; c < I->n_demands; ++c)
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) pd[r] = c;
    int64_t maxne = 0;
    for (int e = 0; e < E; ++e) if (T.off[e + 1] - T.off[e] > maxne) maxne = T.off[e + 1] - T.off[e];
    or_keyed* eb = (or_keyed*)malloc(sizeof(or_keyed) * (size_t)(maxne > 0 ? maxne : 1));
    for (int e = 0; e < E; ++e) {
        double Ve = L[e] - I->cap[e];
        if (!(Ve > 0.0)) continue;
        const int64_t n = T.off[e + 1] - T.off[e];
        for (int64_t j = 0; j < n; ++j) {
            const int64_t r = T.path[T.off[e] + j];
            eb[j].key = log_score(S[pd[r]], Cp[r], alpha);
            eb[j].path = r;
        }
        qsort(eb, (size_t)n, sizeof(or_keyed), keyed_cmp);
        for (int64_t j = 0; j < n && Ve > 0.0; ++j) {
            const int64_t r = eb[j].path;
            const double dx = fmin(x[r], Ve);
            if (dx > trim[r]) trim[r] = dx;
            Ve -= dx;
        }
    }
    for (int64_t r = 0; r < P; ++r) x[r] -= trim[r];
    free(eb); free(trim); free(pd);
    csc_free(&T);
    free(S); free(L); free(Cp);
}

/* ------------------------------------------------------------------ */
/* Exact max-min fair rates when every demand has a single path          */
/* (progressive filling, textbook water-filling): all unfrozen demands   */
/* rise together; a demand freezes when it reaches D_c or when an edge   */
/* on its path fills.  Events in increasing level, edges in a binary    */
/* heap keyed by the level at which they fill, (C_e - frozen load) /     */
/* (unfrozen demands through e); stale heap entries are skipped.         */
/* rate[K] out (caller units).  Returns 1 if a demand has != 1 path.    */
/* ------------------------------------------------------------------ */
typedef struct { double key; int e; } or_hent;

static void heap_push(or_hent* h, int64_t* n, double key, int e) {
    int64_t i = (*n)++;
    h[i].key = key; h[i].e = e;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (h[p].key <= h[i].key) break;
        const or_hent t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static or_hent heap_pop(or_hent* h, int64_t* n) {
    const or_hent top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        const int64_t l = 2 * i + 1, r = l + 1;
        int64_t m = i;
        if (l < *n && h[l].key < h[m].key) m = l;
        if (r < *n && h[r].key < h[m].key) m = r;
        if (m == i) break;
        const or_hent t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

static int dbl_idx_cmp(const void* a, const void* b) {
    const or_keyed* p = (const or_keyed*)a;
    const or_keyed* q = (const or_keyed*)b;
    return (p->key > q->key) - (p->key < q->key);
}

int or_maxmin_single_path(const or_instance* I, double* rate) {
    const int E = I->n_edges;
    const int32_t K = I->n_demands;
    for (int32_t c = 0; c < K; ++c) if (I->dpo[c + 1] - I->dpo[c] != 1) return 1;
    or_csc T;
    csc_build(I, &T);  /* edge -> paths; path r is demand r here */
    double* frozen = (double*)calloc((size_t)E, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)E, sizeof(int64_t));
    unsigned char* done = (unsigned char*)calloc((size_t)K, 1);
    unsigned char* full = (unsigned char*)calloc((size_t)E, 1);
    for (int64_t i = 0; i < I->nnz; ++i) cnt[I->pe[i]]++;
    or_hent* heap = (or_hent*)malloc(sizeof(or_hent) * (size_t)(I->nnz + E + 1));
    int64_t hn = 0;
    for (int e = 0; e < E; ++e) if (cnt[e] > 0) heap_push(heap, &hn, I->cap[e] / (double)cnt[e], e);
    or_keyed* dem = (or_keyed*)malloc(sizeof(or_keyed) * (size_t)(K > 0 ? K : 1));
    for (int32_t c = 0; c < K; ++c) { dem[c].key = I->demand[c]; dem[c].path = c; }
    qsort(dem, (size_t)K, sizeof(or_keyed), dbl_idx_cmp);
    int64_t di = 0;
    /* freezes demand c at level t: its edges lose one unfrozen demand */
    #define OR_FREEZE(cc, tt) do { \
        const int32_t c_ = (cc); const double t_ = (tt); \
        done[c_] = 1; rate[c_] = t_; \
        const int64_t r_ = I->dpo[c_]; \
        for (int64_t i_ = I->peo[r_]; i_ < I->peo[r_ + 1]; ++i_) { \
            const int e_ = I->pe[i_]; \
            frozen[e_] += t_; cnt[e_]--; \
            if (cnt[e_] > 0 && !full[e_]) heap_push(heap, &hn, (I->cap[e_] - frozen[e_]) / (double)cnt[e_], e_); \
        } } while (0)
    for (;;) {
        while (di < K && done[dem[di].path]) ++di;
        /* drop stale heap tops (an edge filled, or its key moved) */
        while (hn > 0) {
            const or_hent h = heap[0];
            if (full[h.e] || cnt[h.e] == 0 || h.key != (I->cap[h.e] - frozen[h.e]) / (double)cnt[h.e]) {
                heap_pop(heap, &hn);
                continue;
            }
            break;
        }
        const double te_ = hn > 0 ? heap[0].key : INFINITY;
        const double td = di < K ? dem[di].key : INFINITY;
        if (!(te_ < INFINITY) && !(td < INFINITY)) break;
        if (td <= te_) {
            OR_FREEZE((int32_t)dem[di].path, td);
            continue;
        }
        const or_hent h = heap_pop(heap, &hn);
        full[h.e] = 1;
        for (int64_t i = T.off[h.e]; i < T.off[h.e + 1]; ++i) {
            const int32_t c = (int32_t)T.path[i];
            if (!done[c]) OR_FREEZE(c, h.key);
        }
    }
    #undef OR_FREEZE
    free(frozen); free(cnt); free(done); free(full); free(heap); free(dem);
    csc_free(&T);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Proportional feasibility scaling -- not in the paper: an alternative  */
/* to Algorithm 2 that scales instead of trimming, so that no demand    */
/* with a positive rate loses all of it.  x[P] in/out (units of cap and  */
/* demand):                                                              */
/*   1. x <- max(x, 0)                                                   */
/*   2. every path of a demand with S_c > D_c is scaled by D_c / S_c     */
/*   3. with L_e the loads after step 2 and f_e = min(1, C_e / L_e),     */
/*      every path is scaled by the smallest f_e over its edges          */
/* After step 3, L_e' <= f_e L_e <= C_e and S_c' <= S_c <= D_c.          */
/* ------------------------------------------------------------------ */
void or_project_scale(const or_instance* I, double* x) {
    const int E = I->n_edges;
    const int64_t P = I->n_paths;
    for (int64_t r = 0; r < P; ++r) if (!(x[r] > 0.0)) x[r] = 0.0;
    for (int32_t c = 0; c < I->n_demands; ++c) {
        double S = 0.0;
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) S += x[r];
        if (S > I->demand[c]) {
            const double g = I->demand[c] / S;
            for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) x[r] *= g;
        }
    }
    double* L = (double*)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    for (int64_t r = 0; r < P; ++r)
        for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) L[I->pe[i]] += x[r];
    for (int e = 0; e < E; ++e) L[e] = (L[e] > I->cap[e]) ? I->cap[e] / L[e] : 1.0;  /* f_e */
    for (int64_t r = 0; r < P; ++r) {
        double g = 1.0;
        for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) g = fmin(g, L[I->pe[i]]);
        x[r] *= g;
    }
    free(L);
}

/* ------------------------------------------------------------------ */
/* Duality gap of a feasible allocation x (caller units).               */
/* For any edge prices p >= 0 the Lagrangian dual                        */
/*   g(p) = sum_e p_e C_e + sum_c max_{0<=S<=D_c} [U(S) - pi_c S],        */
/*   pi_c = min_{r in P_c} sum_{e in r} p_e,                              */
/* bounds the optimum from above (weak duality; Slater's point of         */
/* Appendix C gives strong duality).  Returns gap = g(p) - sum_c U(S_c)   */
/* and writes primal and dual values.                                     */
/* ------------------------------------------------------------------ */
static double conj_term(double D, double pi, double alpha) {
    /* max over 0 <= S <= D of U_alpha(S) - pi S */
    double S;
    if (alpha == 0.0) S = pi < 1.0 ? D : 0.0;
    else if (pi <= 0.0) S = D;
    else {
        const double s_free = exp(-log(pi) / alpha);
        S = s_free < D ? s_free : D;
    }
    if (S <= 0.0) return or_utility(0.0, alpha);
    return or_utility(S, alpha) - pi * S;
}

double or_gap(const or_instance* I, const double* x, const double* p, double alpha, double* primal,
              double* dual) {
    double pr = 0.0, du = 0.0;
    for (int e = 0; e < I->n_edges; ++e) du += p[e] * I->cap[e];
    for (int32_t c = 0; c < I->n_demands; ++c) {
        double S = 0.0, pi = INFINITY;
        for (int64_t r = I->dpo[c]; r < I->dpo[c + 1]; ++r) {
            S += x[r];
            double q = 0.0;
            for (int64_t i = I->peo[r]; i < I->peo[r + 1]; ++i) q += p[I->pe[i]];
            if (q < pi) pi = q;
        }
        pr += or_utility(S, alpha);
        du += conj_term(I->demand[c], pi, alpha);
    }
    if (primal) *primal = pr;
    if (dual) *dual = du;
    return du - pr;
}

/*
 * te.h -- C-ABI of the GATE traffic-engineering iteration engine (libte.so).
 *
 * The library solves path-based alpha-fair traffic engineering (GATE,
 * Section 3.1): given directed edge capacities C_e, demands D_c and a set of
 * pre-computed paths per demand, it finds path rates x_r that maximise
 *     sum_c U_alpha(S_c),   S_c = sum_{r in P_c} x_r            (Eq. 4)
 * subject to S_c <= D_c (Eq. 1), sum_{r ni e} x_r <= C_e (Eq. 2), x >= 0
 * (Eq. 3); alpha = 0 is total throughput, alpha = 1 proportional fairness and
 * alpha -> infinity max-min fairness (Table 3).  It runs the ADMM iteration of
 * Algorithm 1 (Sections 3.2-3.4) on one CUDA device: per-demand rate updates
 * (Eq. 14 with the sum computation of Appendix B.2), per-edge price updates
 * (Eqs. 9, 13), residuals (Eqs. 15-16), residual balancing (Eq. 17), the stop
 * rule (Eq. 18) and alpha-continuation (Section 3.4), followed on request by
 * the feasibility projection of Algorithm 2 (Section 3.5).
 *
 * Conventions for every entry point:
 *  - Status codes are returned; nothing is thrown across the ABI.  A failing
 *    call leaves the handle's last consistent state and stores a message
 *    readable with te_last_error().
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the device that was current at te_create.
 *  - A handle is used by one host thread at a time and issues all its work
 *    on the stream given in te_options.cuda_stream (NULL: the legacy default
 *    stream).  Calls that return values synchronise that stream.
 *  - Units: rates, demands and capacities are in the caller's units.  The
 *    iteration itself runs on values divided by one positive scale (the
 *    geometric mean of the demands by default; see scale_mode), which leaves
 *    the alpha-fair optimum unchanged; te_solve_result reports beta in those
 *    normalised units.
 */
#ifndef TE_H_
#define TE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct te_handle te_handle;

typedef enum {
    TE_OK = 0,
    TE_EINVAL = 1,        /* invalid argument or instance (message says which) */
    TE_ENOMEM = 2,        /* host or device allocation failed                  */
    TE_ECUDA = 3,         /* a CUDA runtime call failed                        */
    TE_ETIMEOUT = 4,      /* a bounded device-side wait gave up; state kept    */
    TE_ENUMERIC = 5,      /* a residual became NaN/Inf                         */
    TE_ENOTCONVERGED = 6, /* reserved                                          */
    TE_EUNSUPPORTED = 7   /* instance exceeds a documented limit               */
} te_status;

/* Directed topology.  edge_src/edge_dst may be NULL (then paths are not
 * checked for being walks). */
typedef struct {
    int32_t n_nodes;
    int32_t n_edges;
    const int32_t* edge_src; /* host [n_edges] */
    const int32_t* edge_dst; /* host [n_edges] */
} te_topology;

/* Pre-computed path sets in CSR form (Section 3.1, "Variables"): demand c
 * owns paths demand_path_off[c] .. demand_path_off[c+1]-1, path r traverses
 * edges path_edges[path_edge_off[r] .. path_edge_off[r+1]-1] in order.
 * demand_src/demand_dst may be NULL (then the walk check is skipped). */
typedef struct {
    int32_t n_demands;
    int32_t pad_;
    int64_t n_paths;
    int64_t nnz;
    const int32_t* demand_src;       /* host [n_demands]   */
    const int32_t* demand_dst;       /* host [n_demands]   */
    const int64_t* demand_path_off;  /* host [n_demands+1] */
    const int64_t* path_edge_off;    /* host [n_paths+1]   */
    const int32_t* path_edges;       /* host [nnz]         */
} te_paths;

/* Solver options; te_default_options() fills the paper's defaults. */
typedef struct {
    double alpha_target;  /* fairness level; INFINITY = max-min (default)      */
    double alpha_start;   /* first alpha of the continuation (default 0)       */
    double alpha_step;    /* continuation increment (default 1, Algorithm 1)   */
    double alpha_max;     /* continuation cap (default 32)                     */
    double gamma;         /* stop threshold on relative r and s (default 1e-3,
                             Section 3.7); negative: never stop early          */
    double gamma_max;     /* > 0: a level of the continuation also counts as
                             converged (Eq. 18) only while the primal residual
                             in the max norm, the largest relative capacity
                             violation max_e n_e |u_e' - u_e| / C_e, is at or
                             below gamma_max; <= 0 (default): off             */
    double A;             /* residual balancing ratio (default 10, Eq. 17)     */
    double C;             /* residual balancing factor (default 2, Eq. 17)     */
    double beta0;         /* initial penalty in normalised units; <= 0
                             (default) picks 1 / (mean path length * mean
                             initial path rate), so the first utility push
                             lambda/(beta n_r) at lambda = 1 equals the mean
                             initial rate                                      */
    double beta_max;      /* > 0: residual balancing never raises beta above
                             beta_max * beta0 (the balancing of Eq. 17 with
                             the paper's residuals can raise beta without
                             bound after alpha increments, which freezes the
                             iterate); 0 (default): no bound                  */
    double balance_floor; /* residual balancing (Eq. 17) acts only while
                             max(r, s) > balance_floor (default 1e-6): below
                             it both residuals of the FP32 iteration are
                             rounding noise and their ratio says nothing.
                             beta also stays within [1e-30, 1e30] (normalised
                             units), where 1/beta is a finite FP32 value      */
    int32_t adapt_beta;   /* 1: residual balancing on (default 1)              */
    int32_t continuation; /* 1: stop when converged on the first iteration
                             after an alpha increment (default 1)              */
    int32_t scale_mode;   /* unit of the normalised problem: 0 = max_e C_e,
                             1 = geometric mean of the demands (default), so
                             the marginal utility S^-alpha of a typical demand
                             stays near 1 as alpha grows; 2 = 1 (caller units) */
    int32_t wait_timeout_ms; /* bound on every grid-wide wait inside te_solve;
                             0 = default (2000 ms)                             */
    int32_t test_withhold_cta; /* test hook for the bounded-wait path: 1 + the
                             index of a CTA that never arrives at the grid
                             barrier, so te_solve must return TE_ETIMEOUT;
                             0 = off (default)                                 */
    int32_t deterministic; /* 1 (default): the edge loads L_e of Eq. 9 are
                             exact integer sums of fixed-point rates, so a run
                             is bit-identical for a given instance and device;
                             0: one FP32 shared-memory add per path-edge
                             incidence instead of two integer adds (the loads,
                             and so the iterates, may differ in the last bits
                             between runs; measured slower on B300, where an
                             FP32 shared atomic costs more than two integer ones) */
    int32_t precision;    /* arithmetic of the iteration: TE_PRECISION_FP32
                             (the only value; FP32 rates and prices, FP64
                             residual sums, gap and stop test)                */
    int32_t edge_mode;    /* where the iteration kernel keeps each CTA's copy
                             of the per-edge arrays (gather weights w_e and the
                             load histogram of Eq. 9): TE_EDGES_AUTO (0,
                             default) shared memory when they fit (about
                             10,770 edges), else global memory (L2);
                             TE_EDGES_GLOBAL (1) global memory always.  Both
                             give the same bits; the global mode takes one
                             64-bit L2 reduction per path-edge incidence
                             instead of two shared-memory atomics and needs
                             deterministic = 1 (else TE_EUNSUPPORTED); above
                             65,534 edges (32-bit ids) it is the only mode   */
    void* cuda_stream;    /* cudaStream_t to run on; NULL = default stream     */
} te_options;

/* te_options.precision */
enum {
    TE_PRECISION_FP32 = 0  /* FP32 iterates (Algorithm 1's rates, prices, per-
                              demand multipliers); the residual norms (Eqs.
                              15-16), their cross-CTA sums, the balancing and
                              stop decisions (Eqs. 17-18) and the gap in FP64 */
};

/* te_options.edge_mode */
enum {
    TE_EDGES_AUTO = 0,   /* shared memory when the per-edge arrays fit, else global */
    TE_EDGES_GLOBAL = 1  /* global memory (L2) always                             */
};

/* Outcome of a te_solve call. */
typedef struct {
    int64_t iters;        /* iterations run by this call                       */
    int64_t total_iters;  /* iterations since te_create / te_reset             */
    double r;             /* last relative primal residual (Eq. 16)            */
    double s;             /* last relative dual residual (Eq. 15)              */
    double beta;          /* penalty after the last iteration (normalised)     */
    double alpha;         /* fairness level after the last iteration           */
    int32_t converged;    /* 1: the stop rule fired in this call               */
    int32_t stop_reason;  /* 0 none, 4 target alpha reached, 8 stagnation after
                             an increment, 16 alpha_max reached                */
} te_solve_result;

/* Fills *opt with the defaults listed above. */
void te_default_options(te_options* opt);

/* Validates the instance, builds the device layout, copies everything to
 * the device and sets the initial state (Algorithm 1: x_r = D_c/|P_c|, all
 * duals zero, alpha = alpha_start).  The caller keeps ownership of every
 * input buffer (they are copied).  demands: host [n_demands], finite and
 * > 0; capacities: host [n_edges], finite and >= 0, and > 0 on every edge
 * used by a path (Slater's condition, Appendix C).  Limits: at most 32 paths
 * per demand, at most 255 edges per path.  Above about 10,770 edges the
 * per-edge arrays of the iteration kernel no longer fit a CTA's shared
 * memory and it keeps them in global memory (edge_mode; such instances need
 * deterministic = 1); above 65,534 edges the device layout stores 32-bit
 * edge ids instead of 16-bit ones, up to about 490,000 edges (each CTA's
 * slice of the prices must fit shared memory beside the staging buffers;
 * more return TE_EUNSUPPORTED).  On success *out
 * receives a new handle.  Errors: TE_EINVAL (bad input; message names the
 * first offending index), TE_EUNSUPPORTED, TE_ENOMEM, TE_ECUDA. */
te_status te_create(const te_topology* topo, const te_paths* paths, const double* demands,
                    const double* capacities, const te_options* opt, te_handle** out);

/* Runs up to max_iters iterations of Algorithm 1 from the current state in
 * one persistent kernel launch, stopping early when the stop rule fires
 * (Eq. 18 with alpha-continuation).  tol is the threshold gamma of Eq. 18
 * for this call (the residuals r and s at or below it count as converged,
 * for the stop and for alpha increments); tol < 0 uses te_options.gamma.
 * tol = 0 runs max_iters iterations unless both residuals are exactly zero.
 * Every step of the iteration runs on the device; the call synchronises and
 * fills *out (may be NULL).  Errors: TE_EINVAL (max_iters < 0 or tol NaN),
 * TE_ETIMEOUT (a grid-wide wait exceeded its limit; the state of the last
 * completed iteration is kept), TE_ENUMERIC, TE_ECUDA. */
te_status te_solve(te_handle* h, int64_t max_iters, double tol, te_solve_result* out);

/* Feasibility step applied by te_allocation. */
enum {
    TE_PROJECT_NONE = 0,  /* the raw iterate (may violate S_c <= D_c, L_e <= C_e) */
    TE_PROJECT_ALG2 = 1,  /* Algorithm 2: non-negativity, demand trims, capacity
                             trims of whole paths in descending S_c^alpha * C_p */
    TE_PROJECT_SCALE = 2  /* not in the paper: non-negativity, each over-served
                             demand scaled to D_c, then each path scaled by the
                             smallest min(1, C_e / L_e) over its edges; never
                             empties a demand that has a positive rate */
};

/* Writes the current rates in the caller's path order and units to x_out
 * [n_paths] (FP32).  project (TE_PROJECT_*) selects the feasibility step,
 * applied to a copy; the iterate itself is not changed.  Both feasibility
 * steps sum in FP64 and round their trims and factors toward zero, so the
 * FP32 result satisfies the constraints up to the FP32 rounding of the
 * conversion to caller units.  out_is_device selects whether x_out is a
 * device or a host pointer.  With TE_PROJECT_ALG2 the handle keeps a list of
 * the violated path-edge incidences (16 bytes each), allocated on the first
 * call that needs it, grown when a later call needs more and freed by
 * te_destroy (so the call may allocate device memory; te_gap and
 * te_gap_projected with TE_PROJECT_ALG2 as well).  Errors: TE_EINVAL (NULL
 * pointer, unknown project), TE_ECUDA (also when that list cannot be
 * allocated). */
te_status te_allocation(te_handle* h, float* x_out, int32_t project, int32_t out_is_device);

/* Duality gap of the projected allocation x^ (caller units, FP64): the
 * Lagrangian dual bound g(p) = sum_e p_e C_e + sum_c max_{0<=S<=D_c}
 * [U_alpha(S) - pi_c S], pi_c = min_{r in P_c} sum_{e in r} p_e, at the
 * current prices p_e = beta u_e, minus sum_c U_alpha(S_c(x^)), at the
 * current alpha (weak duality of the TE problem, Eqs. 1-4; tight at the
 * optimum by Slater's condition, Appendix C).  x^ is the iterate after
 * Algorithm 2 (Section 3.5).  Any output pointer may be NULL. */
te_status te_gap(te_handle* h, double* gap_out, double* primal_out, double* dual_out);

/* te_gap with the feasibility step chosen by project: TE_PROJECT_ALG2
 * (the same as te_gap) or TE_PROJECT_SCALE (proportional scaling, see
 * te_allocation).  Algorithm 2 trims whole paths and can leave a demand at
 * S_c = 0, where U_alpha is -infinity for alpha >= 1 (the primal is then
 * -INFINITY and the gap +INFINITY); scaling keeps every demand that has a
 * rate, so its primal stays finite.  Errors: TE_EINVAL (NULL handle,
 * another project value), TE_ECUDA. */
te_status te_gap_projected(te_handle* h, int32_t project, double* gap_out, double* primal_out,
                           double* dual_out);

/* Current edge prices p_e = beta u_e in the caller's units (FP64,
 * [n_edges]); these are the capacity multipliers dual_cap_e of Eq. 9. */
te_status te_prices(te_handle* h, double* p_out, int32_t out_is_device);

/* Replaces the rates by x0 (caller order and units, [n_paths], FP32) for a
 * warm start (Algorithm 1, optional input x^0).  keep_duals = 0 also resets
 * the prices and alpha to their initial values. */
te_status te_set_warm_start(te_handle* h, const float* x0, int32_t in_is_device, int32_t keep_duals);

/* Replaces the demands D_c (caller order and units, [n_demands], FP64,
 * finite and > 0) without rebuilding the instance, for re-solving as demands
 * drift (Section 2 "Background": TE re-runs on every new demand matrix).
 * in_is_device selects a device or host pointer.  The iterate, prices and
 * alpha are kept (a warm start from the previous allocation); call te_reset
 * for a cold start.  Errors: TE_EINVAL if a demand is not finite and > 0
 * (nothing is changed then). */
te_status te_set_demands(te_handle* h, const double* demands, int32_t in_is_device);

/* Replaces the capacities C_e (edge order and caller units, [n_edges],
 * FP64, finite and >= 0) without rebuilding the instance: a link failure is
 * a capacity of 0 (its paths' rates go to 0 in the limit), a repair or an
 * upgrade a new value (Section 2: TE re-runs when the network changes).
 * in_is_device selects a device or host pointer.  The iterate, prices and
 * alpha are kept (a warm start); call te_reset for a cold start.  Errors:
 * TE_EINVAL if a capacity is not finite and >= 0 (nothing is changed then). */
te_status te_set_capacities(te_handle* h, const double* capacities, int32_t in_is_device);

/* Returns to the initial state of te_create. */
te_status te_reset(te_handle* h);

/* Per-iteration telemetry since the last te_create/te_reset: rows of five
 * doubles (r, s, beta, alpha, event bits: 1 beta changed, 2 alpha
 * incremented, 4/8/16 stop reasons).  Copies min(max_rows, available) rows
 * to host out and returns that count in *rows. */
te_status te_trace(te_handle* h, double* out, int64_t max_rows, int64_t* rows);

/* Sizes of the device layout: n_demands, n_paths, nnz, padded id rows,
 * slots, id width in bytes, persistent grid size, bytes the iteration kernel
 * reads and writes per iteration (the algorithmic traffic), device memory
 * held, and the number of kernels launched through this handle. */
typedef struct {
    int64_t n_demands, n_paths, nnz;
    int64_t id_rows, slots;
    int32_t id_bytes, grid;
    int64_t bytes_per_iter;
    int64_t device_bytes;
    int64_t kernel_launches;  /* kernels this handle has launched so far */
    int32_t edges_global;     /* 1: the iteration kernel keeps its per-edge
                                 arrays in global memory (te_options.edge_mode
                                 asked for it, or they exceed shared memory) */
    int32_t reserved;
} te_layout_info;
te_status te_layout(const te_handle* h, te_layout_info* info);

/* Gradient of the fairness objective through K iterations (not in the
 * paper: the differentiated form, for capacity planning).  From the initial
 * state of Algorithm 1 the handle runs K iterations with beta and alpha fixed
 * (the handle must have been created with adapt_beta = 0, continuation = 0,
 * gamma < 0 and alpha_start = alpha_target finite; else TE_EINVAL) and
 *   J = sum_c U_alpha(S_c^K),   S_c^K = the demand totals after K iterations,
 * then returns J (J_out may be NULL) and dJ/dC_e [n_edges], dJ/dD_c
 * [n_demands] in caller units (FP64; out_is_device selects device or host
 * buffers), by a hand-written reverse pass over the K iterations: the
 * iterate's state is kept every checkpoint_every iterations and each segment
 * is recomputed forward before it is reversed.  The normalisation unit is
 * held fixed (create with scale_mode 2 for caller units, so that the
 * function differentiated does not move the unit).  Forward states are the
 * FP32 iterates; adjoints are FP64.  J is summed in a fixed order and the
 * per-edge weight adjoints as exact 64-bit fixed-point integers (each term
 * rounded to a power-of-two grid set by the step's largest term, about 2^-46
 * of it on the 200-node workload), so a call returns the same bits every
 * time.  Uses device memory of about
 * (K/checkpoint_every + checkpoint_every + 2) times the iterate (released
 * before returning).  The handle's state afterwards is that of an
 * intermediate iteration: call te_reset before solving again. */
te_status te_gradient(te_handle* h, int64_t iters, int32_t checkpoint_every, double* J_out, double* dJ_dC,
                      double* dJ_dD, int32_t out_is_device);

/* ---------------------------------------------------------------------- */
/* Batch of instances (what-if scenarios) over one topology                */
/* ---------------------------------------------------------------------- */
/* Many TE instances that share the topology's edge numbering but have their
 * own path sets (e.g. paths through failed links removed), demands and
 * capacities, solved together: each instance runs Algorithm 1 (with the same
 * options) on its own, all in one launch.  With at least twice as many SMs as
 * instances, te_solve's iteration kernel runs them with SMs / n CTAs each;
 * otherwise a batch kernel runs one instance per CTA, captured in a CUDA
 * graph.  Not in the paper, which solves one instance at a time; the
 * per-instance iteration is the same as te_solve's. */
typedef struct te_batch te_batch;

typedef struct {
    int64_t n_instances, n_paths, id_rows;
    int64_t bytes_per_iter;   /* algorithmic traffic of one iteration of every instance */
    int64_t device_bytes, kernel_launches;
    int32_t warps_per_cta, ctas_per_sm;  /* CTA shape chosen by the first te_batch_solve (0 before) */
    int32_t lanes_per_demand;
    int32_t ctas_per_instance;  /* > 0: the instances run in one launch of te_solve's iteration
                                   kernel with this many CTAs each (chosen at te_batch_create
                                   when there are at most half as many instances as SMs);
                                   0: the batch kernel, one instance per CTA */
} te_batch_info_t;

/* Copies n instances (paths[i], demands[i] [paths[i]->n_demands], capacities[i]
 * [topo->n_edges]; the caller keeps its buffers) to the device and sets every
 * instance to the initial state of Algorithm 1.  Inputs must satisfy the rules
 * of te_create (edge ids are range-checked here, path walks are not).  The
 * options apply to every instance (deterministic = 1, beta_max = 0 and
 * TE_PRECISION_FP32 only; others return TE_EUNSUPPORTED); a NULL cuda_stream makes the batch create
 * and own a stream (graph capture needs one).  Errors as te_create. */
te_status te_batch_create(const te_topology* topo, int32_t n, const te_paths* const* paths,
                          const double* const* demands, const double* const* capacities,
                          const te_options* opt, te_batch** out);

/* Runs up to max_iters iterations of every instance (an instance whose stop
 * rule fires stops there) and fills results[i] (may be NULL).  The first call
 * times each candidate CTA shape (warps per CTA, CTAs per SM) on the first
 * iterations and keeps the fastest; results do not depend on the shape.
 * Later calls with the same remaining budget replay a captured graph.
 * Errors: TE_EINVAL, TE_ETIMEOUT, TE_ENUMERIC, TE_ECUDA, TE_EUNSUPPORTED. */
te_status te_batch_solve(te_batch* b, int64_t max_iters, te_solve_result* results);

/* te_allocation for instance i (its paths in the caller's order and units). */
te_status te_batch_allocation(te_batch* b, int32_t i, float* x_out, int32_t project, int32_t out_is_device);

/* Every instance back to the initial state of Algorithm 1. */
te_status te_batch_reset(te_batch* b);

te_status te_batch_info(const te_batch* b, te_batch_info_t* info);
void te_batch_destroy(te_batch* b);
/* Message of the batch's last error (b NULL: of the last failed te_batch_create). */
const char* te_batch_last_error(const te_batch* b);

/* The update equations of Section 3.3 as printed, run on the device as a
 * multi-block iteration: an ablation beside the two-block iteration of
 * te_solve, not a solver.  From Algorithm 1's start (x = D_c/|P_c|, every
 * rate suggestion y_{e,r} = x_r, all duals zero), iters iterations of, in
 * Algorithm 1's order: the dual updates of the demand cap, the capacity,
 * the consensus (one dual per path-edge incidence) and non-negativity
 * (dual-updates-dem/cap/con/neg), the per-incidence cost of penalty-b and
 * the rate suggestion y_{e,r} = [(mean_e cost - cost_{e,r}) / beta]_+, and
 * the rate formula x_r = (Q_r + U'(S)/beta - (S - D_c + dual_dem_c) +
 * dual_neg_r) / (1 + n_r) of eq. rate-computation with the previous y and
 * duals, S solved from its sum over the demand's paths (closed form at
 * alpha = 0, bisection otherwise).  As printed, the capacity and its dual
 * are common to all paths of an edge and cancel in the rate suggestion, so
 * the rates do not see C_e.  Values are normalised by the geometric mean of
 * the demands; FP64 throughout; per-edge sums in a fixed order.  Inputs
 * are host arrays as for te_create (checked the same way); alpha >= 0 the
 * fairness level, beta > 0 the penalty in normalised units; x_out: host
 * [n_paths], the rates in caller units (FP64).  Device memory is allocated
 * for the call and released before it returns; the call synchronises
 * cuda_stream (NULL: default stream).  Errors (message via
 * te_last_error(NULL)): TE_EINVAL, TE_EUNSUPPORTED (more than 2^31 - 1
 * incidences), TE_ENOMEM, TE_ECUDA. */
te_status te_literal_run(const te_topology* topo, const te_paths* paths, const double* demands,
                         const double* capacities, double alpha, double beta, int64_t iters, double* x_out,
                         void* cuda_stream);

/* The duality gap of te_gap for a caller-supplied allocation, computed
 * without allocating any memory (the paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc where they need the
 * gap, such as code inside a memory pool that owns all device memory or a
 * control loop whose allocations are frozen after start-up).
 * Every pointer is a device pointer of the current device, owned by the
 * caller: the instance in the CSR form of te_paths (demand_path_off
 * [n_demands+1], path_edge_off [n_paths+1], path_edges [nnz]), demands
 * [n_demands] and capacities [n_edges] (FP64, caller units), a feasible
 * allocation x [n_paths] (FP32, e.g. from te_allocation with project = 1),
 * edge prices [n_edges] (FP64, e.g. from te_prices) and the fairness level
 * alpha >= 0; out [3] receives {gap, primal, dual} in FP64 as te_gap reports
 * them.  The work is queued on cuda_stream (NULL: default stream) and the
 * call returns without synchronising.
 * Working memory is one static device array of 16384 slots of two doubles
 * (256 KB, held on every device that loads the library until exit), so
 * ceil(n_demands/256) + ceil(n_edges/256) must not exceed 16384 (about 4.19
 * million demands); larger inputs return TE_EUNSUPPORTED before any work is
 * queued.  Nothing in that array has to start at zero.  All calls on a
 * device share it: calls that overlap on the GPU race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Errors: TE_EINVAL (null
 * pointer, bad size, alpha < 0), TE_EUNSUPPORTED (too large), TE_ECUDA. */
te_status te_gap_noalloc(int32_t n_edges, int32_t n_demands, int64_t n_paths, int64_t nnz,
                         const int64_t* demand_path_off, const int64_t* path_edge_off,
                         const int32_t* path_edges, const double* demands, const double* capacities,
                         const float* x, const double* prices, double alpha, double* out,
                         void* cuda_stream);

/* Releases every resource of the handle.  NULL is ignored. */
void te_destroy(te_handle* h);

/* Message of the last failing call on h (never NULL); with h == NULL, the
 * message of the last failing te_create in this thread. */
const char* te_last_error(const te_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* TE_H_ */

// Batch of TE instances on one GPU: many what-if scenarios (failed links,
// perturbed demand matrices) over one topology, solved in one launch.
//
// Every instance has its own path sets, demands and capacities; their sliced
// layouts (see te_internal.cuh) are concatenated, each with instance-local
// indices.  The batch kernel gives a whole instance to one CTA: the CTA holds
// the instance's edge arrays (load histogram, gather weights, prices) in
// shared memory and runs its iterations (Algorithm 1: phase A over the
// instance's blocks, then the per-edge price update, the residuals, residual
// balancing, the stop rule and alpha-continuation) with CTA barriers only.
// CTAs take instances from a global counter, so instances of uneven size and
// uneven iteration counts balance over the SMs, and an instance that stops
// early frees its CTA for the next.  The launch is captured in a CUDA graph
// and replayed on later calls with the same iteration budget.
//
// Results do not depend on the CTA shape: loads are exact integer sums,
// residual terms are stored per block and reduced over a fixed number of
// partial sums in a fixed order.  The first te_batch_solve times the
// candidate CTA shapes on the batch's own first iterations and keeps the
// fastest (these iterations are part of the solve).
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "te.h"
#include "te_kernels.cuh"
#include "te_layout.h"
#include "te_proj.h"

using te::kLanes;

namespace te {
namespace {

constexpr int kRedParts = 256;  // partial sums of every CTA-wide reduction

// One instance of the batch: where its pieces sit in the concatenated arrays.
// Instances with the same path sets (e.g. the demand matrices of one failure
// scenario) share one layout: id rows, block records, slot and row offsets.
struct BatchInst {
    long long row0;   // first id row of its layout
    int meta0;        // first block record of its layout
    int nblocks;
    long long slot0;  // first slot of its rates (x[(slot0 + s) * 32 + lane])
    long long dslot0; // first demand slot of its demands and multipliers
    long long res0;   // first block of its residual terms
};

struct BatchArgs {
    const BatchInst* inst;
    int ninst;
    int E;
    int dpb;
    const uint16_t* ids;
    const BlockMeta* blkmeta;
    const unsigned* hops;  // [blocks*32] hop counts of a lane's paths, slot j in bits 8j..8j+7
    const float* Dn;
    float* lam;
    float* blkres;
    float* x;            // [2][total slots * 32]
    long long xstride;   // total slots * 32
    float* u;            // [ninst][E]
    float* w;            // [ninst][E]
    const float* cap_n;  // [ninst][E]
    const float* ne_f;   // [ninst][E]
    const float* inv_ne; // [ninst][E]
    Scalars* sc;         // [ninst]
    Options o;
    long long max_iters;
    long long timeout_ns;
    int* status;
    unsigned* next;      // instance counter (zeroed before the launch)
};

// Sum over the CTA of a per-thread value held by threads < kRedParts, in a
// fixed order (thread 0 adds the partials in index order): the same for any
// CTA shape.
__device__ double fixed_sum(double v, double* part) {
    __syncthreads();
    if (threadIdx.x < kRedParts) part[threadIdx.x] = v;
    __syncthreads();
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedParts; ++i) t += part[i];
        s_tot = t;
    }
    __syncthreads();
    return s_tot;
}

// Largest per-thread value over the CTA (threads < kRedParts).
__device__ double fixed_max(double v, double* part) {
    __syncthreads();
    if (threadIdx.x < kRedParts) part[threadIdx.x] = v;
    __syncthreads();
    __shared__ double s_max;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedParts; ++i) t = fmax(t, part[i]);
        s_max = t;
    }
    __syncthreads();
    return s_max;
}

template <int G, int W>
__global__ void __launch_bounds__(W * 32) k_batch(BatchArgs a) {
    constexpr int kThreads = W * 32;
    static_assert(kThreads >= kRedParts, "the fixed reductions take one partial per thread");
    extern __shared__ __align__(128) unsigned smem[];
    const int E = a.E;
    unsigned* h_hi = smem;                                   // [E+1]
    unsigned* h_lo = h_hi + (E + 1);                         // [E+1]
    float* w_s = reinterpret_cast<float*>(h_lo + (E + 1));  // [E+1], w_s[E] = 0
    float* s_u = w_s + (E + 1);                              // [E]
    uint16_t* stage = reinterpret_cast<uint16_t*>(smem + ((4 * (size_t)E + 3 + 31) & ~size_t(31)));
    __shared__ double s_part[kRedParts];
    __shared__ int s_inst;

    const int tid = threadIdx.x, warp = tid >> 5;
    WarpStage ws;
    ws.base = stage + (size_t)(warp * 2) * kStageRows * kLanes;
    bool failed = false;
    __syncthreads();

    while (!failed) {
        if (tid == 0) s_inst = (int)atomicAdd(a.next, 1u);
        __syncthreads();
        const int ii = s_inst;
        if (ii >= a.ninst) break;
        const BatchInst I = a.inst[ii];
        const size_t eo = (size_t)ii * E;
        for (int e = tid; e < E; e += kThreads) {
            w_s[e] = a.w[eo + e];
            s_u[e] = a.u[eo + e];
            h_hi[e] = 0u;
            h_lo[e] = 0u;
        }
        if (tid == 0) {
            w_s[E] = 0.f;
            h_hi[E] = 0u;
            h_lo[E] = 0u;
        }
        Scalars sc = a.sc[ii];
        sc.converged = 0;
        sc.stop_reason = 0;
        long long done = 0;
        const BlockCtx bc{a.Dn + I.dslot0, a.lam + I.dslot0, a.blkres + (size_t)I.res0 * 3,
                          a.hops + (size_t)I.meta0 * kLanes, a.dpb, (uint16_t)E};
        const BlockMeta* bm = a.blkmeta + I.meta0;
        const uint16_t* ids = a.ids + (size_t)I.row0 * kLanes;
        const float* cap = a.cap_n + eo;
        const float* nef = a.ne_f + eo;
        const float* inv = a.inv_ne + eo;
        __syncthreads();

        for (long long it = 0; it < a.max_iters; ++it) {
            const float* xin = a.x + (size_t)sc.xbuf * a.xstride + (size_t)I.slot0 * kLanes;
            float* xout = a.x + (size_t)(sc.xbuf ^ 1) * a.xstride + (size_t)I.slot0 * kLanes;
            const float inv_beta = (float)(1.0 / sc.beta);
            const float logbeta = (float)log(sc.beta);
            const float beta_f = (float)sc.beta;
            const float alpha = (float)sc.alpha;
            const float inv_alpha = alpha > 0.f ? 1.f / alpha : 0.f;

            // phase A: the instance's blocks, shared among the warps
            LaneRes unused;
            run_blocks<G, kStageRows, false, true, true>(0, 1, I.nblocks, bm, ids, xin, xout, bc, ws, w_s, h_hi, h_lo, inv_beta,
                                             logbeta, beta_f, alpha, inv_alpha, unused);
            __syncthreads();
            if (*(volatile int*)a.status != 0) failed = true;
            if (__syncthreads_or(failed)) {
                failed = true;
                break;
            }

            // residual terms of the blocks
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            if (tid < kRedParts)
                for (int b = tid; b < I.nblocks; b += kRedParts) {
                    const float* r = bc.blkres + (size_t)b * 3;
                    t0 += (double)__ldcg(&r[0]);
                    t1 += (double)__ldcg(&r[1]);
                    t2 += (double)__ldcg(&r[2]);
                }
            const double v0 = fixed_sum(t0, s_part);
            const double v1 = fixed_sum(t1, s_part);
            const double v2 = fixed_sum(t2, s_part);

            // per-edge price update (Eqs. 9/13 after the per-edge collapse):
            // thread t takes edges t, t + kRedParts, ... (the primal residual
            // partials then do not depend on the CTA shape)
            double r2 = 0.0;
            float vmax = 0.f;  // largest relative capacity violation n_e |d_e| / C_e
            if (tid < kRedParts)
                for (int e = tid; e < E; e += kRedParts) {
                    const float L = (float)((double)h_hi[e] * 0x1p-12 + (double)h_lo[e] * 0x1p-24);
                    h_hi[e] = 0u;
                    h_lo[e] = 0u;
                    const float ne = __ldg(&nef[e]);
                    const float u = s_u[e];
                    float un = 0.f;
                    const float ce = __ldg(&cap[e]);
                    if (ne > 0.f) un = fmaxf(0.f, fmaf(L - ce, __ldg(&inv[e]), u));
                    const float d = un - u;
                    r2 += (double)(ne * d * d);
                    if (ne > 0.f) vmax = fmaxf(vmax, __fdiv_ru(ne * fabsf(d), ce));
                    s_u[e] = un;
                    w_s[e] = un + d;
                }
            const double v3 = fixed_sum(r2, s_part);
            const double v4 = fixed_max((double)vmax, s_part);

            // control: residuals, beta, alpha, stop (identical in every thread)
            const double s_res = sqrt(v0) / fmax(sqrt(v1), 1e-30);
            const double r_res = sqrt(v3) / fmax(sqrt(v2), 1e-30);
            sc.xbuf ^= 1;
            sc.iter_total++;
            sc.iter_alpha++;
            done++;
            const bool numeric_ok = isfinite(s_res) && isfinite(r_res);
            if (numeric_ok && a.o.adapt_beta && fmax(r_res, s_res) > a.o.balance_floor) {
                const double nb = balanced_beta(sc.beta, r_res, s_res, a.o.A, a.o.C, a.o.beta_cap);
                if (nb != sc.beta) {
                    // scaled prices follow beta; the weights keep d: w = u' ratio + d
                    const float ratio = (float)(sc.beta / nb);
                    sc.beta = nb;
                    for (int e = tid; e < E; e += kThreads) {
                        const float un = s_u[e];
                        w_s[e] = fmaf(un, ratio - 1.f, w_s[e]);
                        s_u[e] = un * ratio;
                    }
                }
            }
            sc.r = r_res;
            sc.s = s_res;
            if (!numeric_ok) {
                if (tid == 0) atomicCAS(a.status, 0, kStatusNumeric);
                failed = true;
                break;
            }
            bool stop = false;
            int event = 0;
            if (r_res <= a.o.gamma && s_res <= a.o.gamma && (a.o.gamma_max <= 0.0 || v4 <= a.o.gamma_max)) {
                if (sc.alpha >= a.o.alpha_target) {
                    stop = true; event = 4;
                } else if (a.o.continuation && sc.iter_alpha == 1 && sc.alpha > a.o.alpha_start) {
                    stop = true; event = 8;
                } else if (sc.alpha >= a.o.alpha_max) {
                    stop = true; event = 16;
                } else {
                    double na = sc.alpha + a.o.alpha_step;
                    if (na > a.o.alpha_target) na = a.o.alpha_target;
                    if (na > a.o.alpha_max) na = a.o.alpha_max;
                    sc.alpha = na;
                    sc.iter_alpha = 0;
                }
            }
            __syncthreads();
            if (stop) {
                sc.converged = 1;
                sc.stop_reason = event;
                break;
            }
        }
        __syncthreads();
        for (int e = tid; e < E; e += kThreads) {
            a.u[eo + e] = s_u[e];
            a.w[eo + e] = w_s[e];
        }
        if (tid == 0) {
            sc.iters_run = done;
            a.sc[ii] = sc;
        }
        __syncthreads();
    }
}

size_t batch_smem_bytes(int E, int W) {
    size_t b = ((4 * (size_t)E + 3 + 31) & ~size_t(31)) * sizeof(unsigned);
    b += (size_t)W * 2 * kStageRows * kLanes * sizeof(uint16_t);
    return b;
}

template <int G, int W>
cudaError_t launch_batch_t(const BatchArgs& a, int ctas_per_sm, int nsm, cudaStream_t st) {
    const size_t smem = batch_smem_bytes(a.E, W);
    cudaError_t err = cudaFuncSetAttribute(k_batch<G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int grid = std::max(1, std::min(a.ninst, nsm * ctas_per_sm));
    k_batch<G, W><<<grid, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int G, int W>
cudaError_t batch_occupancy_t(int E, int* blocks) {
    const size_t smem = batch_smem_bytes(E, W);
    cudaError_t err = cudaFuncSetAttribute(k_batch<G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch<G, W>, W * 32, smem);
}

// CTA shapes the first solve chooses from: warps per CTA (8 or 16).
constexpr int kShapes[2] = {8, 16};

cudaError_t launch_batch(int G, int W, const BatchArgs& a, int ctas_per_sm, int nsm, cudaStream_t st) {
#define TE_BATCH_CASE(g, w) \
    if (G == g && W == w) return launch_batch_t<g, w>(a, ctas_per_sm, nsm, st);
    TE_BATCH_CASE(1, 8) TE_BATCH_CASE(1, 16) TE_BATCH_CASE(2, 8) TE_BATCH_CASE(2, 16)
    TE_BATCH_CASE(4, 8) TE_BATCH_CASE(4, 16) TE_BATCH_CASE(8, 8) TE_BATCH_CASE(8, 16)
#undef TE_BATCH_CASE
    return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int G, int W, int E, int* blocks) {
#define TE_BATCH_CASE(g, w) \
    if (G == g && W == w) return batch_occupancy_t<g, w>(E, blocks);
    TE_BATCH_CASE(1, 8) TE_BATCH_CASE(1, 16) TE_BATCH_CASE(2, 8) TE_BATCH_CASE(2, 16)
    TE_BATCH_CASE(4, 8) TE_BATCH_CASE(4, 16) TE_BATCH_CASE(8, 8) TE_BATCH_CASE(8, 16)
#undef TE_BATCH_CASE
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace te

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct te_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // created when the caller gives no stream
    int n = 0, E = 0, G = 1, dpb = 32, nsm = 0;
    te::Options o{};
    double beta0_opt = 0.0;
    std::vector<double> scale, beta0;   // per instance
    std::vector<te::BatchInst> inst;    // host copy
    std::vector<te::Layout> views;      // per instance, for projection and the gather to caller order
    std::vector<long long> P;           // paths per instance
    long long total_slots = 0, total_blocks = 0, total_rows = 0, total_dslots = 0;
    long long bytes_per_iter = 0, device_bytes = 0, launches = 0;
    long long timeout_ns = 2000000000LL;
    int shape_w = 0, shape_ctas = 0;    // chosen CTA shape (0: not yet tuned)
    // fewer instances than half the SMs: the iteration kernel of te_solve runs
    // them all in one cooperative launch, `group` CTAs per instance (0: the
    // batch kernel, one instance per CTA)
    int group = 0;
    unsigned* hops = nullptr;           // [blocks*32] per layout
    float *u_next = nullptr, *w_next = nullptr;  // [n][E]
    uint2* gloads = nullptr;            // [n][group][E] per-CTA partial loads
    double* gpart = nullptr;            // [n][2][group][kPartWidth]
    unsigned* gbar = nullptr;           // [n] barrier counters
    te::IterArgs* d_args = nullptr;     // [n]
    std::vector<te::IterArgs> h_args;
    std::vector<float> shape_ms;
    std::map<long long, cudaGraphExec_t> graphs;
    std::vector<void*> owned;
    // device
    te::BatchInst* d_inst = nullptr;
    uint16_t* ids = nullptr;
    te::BlockMeta* blkmeta = nullptr;
    unsigned* rowoff = nullptr;
    int* slotbase = nullptr;
    float *Dn = nullptr, *lam = nullptr, *blkres = nullptr, *x = nullptr, *u = nullptr, *w = nullptr;
    float *cap = nullptr, *ne = nullptr, *inv = nullptr;
    unsigned char* np = nullptr;
    int* demand_of = nullptr;
    long long* slot_path = nullptr;
    double* Dc = nullptr;
    te::Scalars* sc = nullptr;
    int* status = nullptr;
    unsigned* next = nullptr;
    float* xtmp = nullptr;
    float* user = nullptr;
    te::ProjScratch ps{};
    std::vector<te::Scalars> hsc;
    std::string err;

    template <typename T>
    cudaError_t alloc(T** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) {
            owned.push_back(q);
            device_bytes += (long long)bytes;
        }
        *p = static_cast<T*>(q);
        return e;
    }
    te_status fail(te_status s, const std::string& m) {
        err = m;
        return s;
    }
    te_status cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return TE_OK;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return TE_ECUDA;
    }
};

namespace {
thread_local std::string g_batch_create_error;
}

extern "C" void te_batch_destroy(te_batch* b) {
    if (!b) return;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (void* p : b->owned) cudaFree(p);
    if (b->ps.vlist) cudaFree(b->ps.vlist);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
}

extern "C" const char* te_batch_last_error(const te_batch* b) {
    if (!b) return g_batch_create_error.c_str();
    return b->err.c_str();
}

extern "C" te_status te_batch_reset(te_batch* b) {
    if (!b) return TE_EINVAL;
    cudaStream_t s = b->stream;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    for (int i = 0; i < b->n; ++i) {
        te::Layout V = b->views[i];
        A(te::launch_init_x(V, b->x + (size_t)b->inst[i].slot0 * kLanes, s));
        b->launches += 1;
    }
    A(cudaMemsetAsync(b->u, 0, sizeof(float) * (size_t)b->n * b->E, s));
    A(cudaMemsetAsync(b->w, 0, sizeof(float) * (size_t)b->n * b->E, s));
    A(cudaMemsetAsync(b->lam, 0, sizeof(float) * (size_t)b->total_dslots, s));
    for (int i = 0; i < b->n; ++i) {
        te::Scalars sc{};
        sc.beta = b->beta0[i];
        sc.alpha = (isfinite(b->o.alpha_target) && b->o.alpha_start > b->o.alpha_target) ? b->o.alpha_target
                                                                                         : b->o.alpha_start;
        b->hsc[i] = sc;
    }
    A(cudaMemcpyAsync(b->sc, b->hsc.data(), sizeof(te::Scalars) * b->n, cudaMemcpyHostToDevice, s));
    A(cudaStreamSynchronize(s));
    return b->cuda(ce, "te_batch_reset");
}

extern "C" te_status te_batch_create(const te_topology* topo, int32_t n, const te_paths* const* paths,
                                     const double* const* demands, const double* const* capacities,
                                     const te_options* opt_in, te_batch** out) {
    g_batch_create_error.clear();
    if (!out || !topo || n <= 0 || !paths || !demands || !capacities) {
        g_batch_create_error = "null argument or empty batch";
        return TE_EINVAL;
    }
    *out = nullptr;
    te_options opt;
    if (opt_in) opt = *opt_in; else te_default_options(&opt);
    if (!(opt.gamma == opt.gamma) || !(opt.balance_floor >= 0.0) || !(opt.C > 1.0) || !(opt.A > 0.0) || (opt.scale_mode != 0 && opt.scale_mode != 1) ||
        !(opt.alpha_step > 0.0) || opt.alpha_start < 0.0 || opt.alpha_target < 0.0 || opt.alpha_max < 0.0 ||
        (opt.deterministic != 0 && opt.deterministic != 1)) {
        g_batch_create_error = "invalid options";
        return TE_EINVAL;
    }
    if (opt.deterministic == 0 || opt.precision != TE_PRECISION_FP32) {
        g_batch_create_error = "the batch engine runs the deterministic FP32 iteration only "
                               "(deterministic = 1, precision = TE_PRECISION_FP32)";
        return TE_EUNSUPPORTED;
    }
    te_batch* b = new (std::nothrow) te_batch();
    if (!b) { g_batch_create_error = "out of host memory"; return TE_ENOMEM; }
    auto bail = [&](te_status s) {
        g_batch_create_error = b->err;
        te_batch_destroy(b);
        return s;
    };
    cudaGetDevice(&b->device);
    b->stream = (cudaStream_t)opt.cuda_stream;
    if (!b->stream) {  // graph capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            b->err = "stream creation failed";
            return bail(TE_ECUDA);
        }
        b->stream = b->own_stream;
    }
    b->n = n;
    b->E = topo->n_edges;
    b->o.alpha_target = opt.alpha_target;
    b->o.alpha_start = opt.alpha_start;
    b->o.alpha_step = opt.alpha_step;
    b->o.alpha_max = opt.alpha_max;
    b->o.gamma = opt.gamma;
    b->o.A = opt.A;
    b->o.C = opt.C;
    b->o.adapt_beta = opt.adapt_beta;
    b->o.balance_floor = opt.balance_floor;
    b->o.gamma_max = opt.gamma_max;
    b->o.beta_cap = 1e30;
    if (opt.beta_max > 0.0) {
        b->err = "beta_max is not supported by the batch engine (per-instance beta0)";
        return bail(TE_EUNSUPPORTED);
    }
    b->o.deterministic = 1;
    b->o.continuation = opt.continuation;
    b->o.withhold_cta = -1;
    if (opt.wait_timeout_ms > 0) b->timeout_ns = (long long)opt.wait_timeout_ms * 1000000LL;
    const int E = b->E;

    // every instance's layout, with a common number of lanes per demand;
    // instances whose paths are the same arrays share one layout
    int kmax = 1;
    for (int i = 0; i < n; ++i) {
        const te_paths* P = paths[i];
        if (!P || P->n_demands <= 0) { b->err = "instance without demands"; return bail(TE_EINVAL); }
        for (int c = 0; c < P->n_demands; ++c)
            kmax = std::max<long long>(kmax, P->demand_path_off[c + 1] - P->demand_path_off[c]);
    }
    int G = 1;
    while (G * te::kMaxPathsPerLane < kmax) G *= 2;
    b->G = G;
    std::vector<int> lay_of(n, -1);  // layout index of each instance
    std::vector<int> lay_first;      // first instance of each layout
    for (int i = 0; i < n; ++i) {
        for (size_t j = 0; j < lay_first.size() && lay_of[i] < 0; ++j) {
            const te_paths* Q = paths[lay_first[j]];
            const te_paths* P = paths[i];
            if (P->n_demands == Q->n_demands && P->n_paths == Q->n_paths && P->nnz == Q->nnz &&
                P->demand_path_off == Q->demand_path_off && P->path_edge_off == Q->path_edge_off &&
                P->path_edges == Q->path_edges)
                lay_of[i] = (int)j;
        }
        if (lay_of[i] < 0) {
            lay_of[i] = (int)lay_first.size();
            lay_first.push_back(i);
        }
    }
    const int nl = (int)lay_first.size();
    b->scale.resize(n);
    b->beta0.resize(n);
    for (int i = 0; i < n; ++i) {
        const te_paths* P = paths[i];
        const double* D = demands[i];
        const double* C = capacities[i];
        const int K = P->n_demands;
        for (int c = 0; c < K; ++c)
            if (!(D[c] > 0.0) || !isfinite(D[c])) { b->err = "a demand is not finite and positive"; return bail(TE_EINVAL); }
        for (int e = 0; e < E; ++e)
            if (!(C[e] >= 0.0) || !isfinite(C[e])) { b->err = "a capacity is not finite and >= 0"; return bail(TE_EINVAL); }
        if (lay_first[lay_of[i]] == i)
            for (long long k = 0; k < P->nnz; ++k)
                if (P->path_edges[k] < 0 || P->path_edges[k] >= E) { b->err = "edge id out of range"; return bail(TE_EINVAL); }
        double scale = 0.0;
        if (opt.scale_mode == 1) {
            double lg = 0.0;
            for (int c = 0; c < K; ++c) lg += log(D[c]);
            scale = exp(lg / (double)K);
        } else {
            for (int e = 0; e < E; ++e) scale = std::max(scale, C[e]);
        }
        b->scale[i] = scale;
        if (opt.beta0 > 0.0) {
            b->beta0[i] = opt.beta0;
        } else {
            double dsum = 0.0;
            for (int c = 0; c < K; ++c) dsum += D[c] / scale;
            const double xbar = dsum / (double)P->n_paths, nbar = (double)P->nnz / (double)P->n_paths;
            b->beta0[i] = 1.0 / (nbar * xbar);
        }
    }
    // layouts built in parallel (each build also spreads its bank balancing)
    std::vector<te::HostLayout> hl(nl);
    std::vector<te_status> lst(nl, TE_OK);
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const int nt = std::max(1, std::min<int>(nl, hw ? (int)std::max(1u, hw / 4) : 1));
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t]() {
                for (int j = t; j < nl; j += nt) {
                    const int i = lay_first[j];
                    lst[j] = te::build_host_layout(topo, paths[i], demands[i], capacities[i], b->scale[i], G, hl[j]);
                }
            });
        for (auto& th : pool) th.join();
    }
    for (int j = 0; j < nl; ++j) {
        if (lst[j] != TE_OK) { b->err = "instance " + std::to_string(lay_first[j]) + ": " + hl[j].err; return bail(lst[j]); }
        if (hl[j].G != G) { b->err = "lanes per demand differ between instances"; return bail(TE_EUNSUPPORTED); }
    }
    b->dpb = hl[0].dpb;
    // where each layout sits
    std::vector<long long> lrow0(nl), lro(nl), lso(nl);
    std::vector<int> lmeta0(nl);
    long long rows = 0, ro = 0, so = 0, lslots = 0;
    int metas = 0;
    std::vector<long long> lslot0(nl);
    for (int j = 0; j < nl; ++j) {
        lrow0[j] = rows;
        lmeta0[j] = metas;
        lro[j] = ro;
        lso[j] = so;
        lslot0[j] = lslots;
        rows += hl[j].nrows;
        metas += hl[j].nblocks;
        ro += (long long)hl[j].rowoff.size();
        so += (long long)hl[j].slotbase.size();
        lslots += hl[j].nslots;
    }
    // where each instance's state sits
    b->inst.resize(n);
    b->P.resize(n);
    long long slots = 0, dslots = 0, res = 0;
    for (int i = 0; i < n; ++i) {
        const int j = lay_of[i];
        b->inst[i] = te::BatchInst{lrow0[j], lmeta0[j], hl[j].nblocks, slots, dslots, res};
        b->P[i] = hl[j].P;
        slots += hl[j].nslots;
        dslots += (long long)hl[j].nblocks * b->dpb;
        res += hl[j].nblocks;
    }
    b->total_rows = rows;
    b->total_slots = slots;
    b->total_blocks = res;
    b->total_dslots = dslots;

    int nsm = 0;
    if (b->cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device), "device query"))
        return bail(TE_ECUDA);
    b->nsm = nsm;
    if (te::batch_smem_bytes(E, 8) > 227 * 1024) {
        b->err = "too many edges for the batch kernel's shared memory";
        return bail(TE_EUNSUPPORTED);
    }

    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    size_t maxP = 0, maxND = 0, maxNS = 0;
    for (int j = 0; j < nl; ++j) {
        maxP = std::max<size_t>(maxP, (size_t)hl[j].P);
        maxND = std::max<size_t>(maxND, (size_t)hl[j].nblocks * b->dpb);
        maxNS = std::max<size_t>(maxNS, (size_t)hl[j].nslots * kLanes);
    }
    A(b->alloc(&b->d_inst, sizeof(te::BatchInst) * n));
    A(b->alloc(&b->ids, sizeof(uint16_t) * (size_t)rows * kLanes));
    A(b->alloc(&b->blkmeta, sizeof(te::BlockMeta) * (size_t)metas));
    A(b->alloc(&b->rowoff, sizeof(unsigned) * (size_t)ro));
    A(b->alloc(&b->slotbase, sizeof(int) * (size_t)so));
    A(b->alloc(&b->np, (size_t)metas * b->dpb));
    A(b->alloc(&b->demand_of, sizeof(int) * (size_t)metas * b->dpb));
    A(b->alloc(&b->slot_path, sizeof(long long) * (size_t)lslots * kLanes));
    A(b->alloc(&b->Dn, sizeof(float) * (size_t)dslots));
    A(b->alloc(&b->Dc, sizeof(double) * (size_t)dslots));
    A(b->alloc(&b->lam, sizeof(float) * (size_t)dslots));
    A(b->alloc(&b->blkres, sizeof(float) * 3 * (size_t)res));
    A(b->alloc(&b->x, sizeof(float) * 2 * (size_t)slots * kLanes));
    A(b->alloc(&b->u, sizeof(float) * (size_t)n * E));
    A(b->alloc(&b->w, sizeof(float) * (size_t)n * E));
    A(b->alloc(&b->cap, sizeof(float) * (size_t)n * E));
    A(b->alloc(&b->ne, sizeof(float) * (size_t)n * E));
    A(b->alloc(&b->inv, sizeof(float) * (size_t)n * E));
    A(b->alloc(&b->sc, sizeof(te::Scalars) * n));
    A(b->alloc(&b->status, sizeof(int)));
    A(b->alloc(&b->next, sizeof(unsigned)));
    A(b->alloc(&b->xtmp, sizeof(float) * maxNS));
    A(b->alloc(&b->user, sizeof(float) * maxP));
    A(b->alloc(&b->ps.S, sizeof(double) * maxND));
    A(b->alloc(&b->ps.loads, sizeof(unsigned long long) * E));
    A(b->alloc(&b->ps.viol, (size_t)E));
    A(b->alloc(&b->ps.vidx, sizeof(int) * E));
    A(b->alloc(&b->ps.nviol, sizeof(int)));
    A(b->alloc(&b->ps.hist, sizeof(unsigned long long) * 256 * (size_t)E));
    A(b->alloc(&b->ps.prefix, sizeof(unsigned long long) * E));
    A(b->alloc(&b->ps.rem, sizeof(double) * E));
    A(b->alloc(&b->ps.Cp, maxNS));
    A(b->alloc(&b->ps.score, sizeof(double) * (maxND + 256)));
    A(b->alloc(&b->ps.vtotal, 3 * sizeof(unsigned long long)));
    A(b->alloc(&b->hops, sizeof(unsigned) * (size_t)metas * kLanes));
    // one cooperative launch of the iteration kernel with `group` CTAs per
    // instance when there are fewer instances than half the SMs (one
    // instance per CTA would leave SMs idle)
    if (2 * n <= nsm) {
        const int g = nsm / n;
        int occ = 0;
        if (te::iter_smem_bytes(E, g, true) <= 227 * 1024 &&
            te::iter_occupancy(G, true, E, g, &occ) == cudaSuccess && occ >= 1)
            b->group = g;
        cudaGetLastError();
    }
    if (b->group > 0) {
        const size_t g = (size_t)b->group;
        A(b->alloc(&b->u_next, sizeof(float) * (size_t)n * E));
        A(b->alloc(&b->w_next, sizeof(float) * (size_t)n * E));
        A(b->alloc(&b->gloads, sizeof(uint2) * (size_t)n * g * E));
        A(b->alloc(&b->gpart, sizeof(double) * (size_t)n * 2 * g * te::kPartWidth));
        A(b->alloc(&b->gbar, sizeof(unsigned) * (size_t)n));
        A(b->alloc(&b->d_args, sizeof(te::IterArgs) * (size_t)n));
    }
    if (ce != cudaSuccess) {
        b->err = std::string("device allocation failed: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return bail(ce == cudaErrorMemoryAllocation ? TE_ENOMEM : TE_ECUDA);
    }
    cudaStream_t s = b->stream;
    A(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(te::BatchInst) * n, cudaMemcpyHostToDevice, s));
    for (int j = 0; j < nl; ++j) {
        const te::HostLayout& H = hl[j];
        const size_t nd = (size_t)H.nblocks * b->dpb;
        A(cudaMemcpyAsync(b->ids + (size_t)lrow0[j] * kLanes, H.ids.data(), sizeof(uint16_t) * H.ids.size(),
                          cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->blkmeta + lmeta0[j], H.blkmeta.data(), sizeof(te::BlockMeta) * H.nblocks,
                          cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->rowoff + lro[j], H.rowoff.data(), sizeof(unsigned) * H.rowoff.size(), cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->slotbase + lso[j], H.slotbase.data(), sizeof(int) * H.slotbase.size(), cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->hops + (size_t)lmeta0[j] * kLanes, H.hops.data(), sizeof(unsigned) * H.hops.size(),
                          cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->np + (size_t)lmeta0[j] * b->dpb, H.np.data(), nd, cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->demand_of + (size_t)lmeta0[j] * b->dpb, H.demand_of.data(), sizeof(int) * nd,
                          cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->slot_path + (size_t)lslot0[j] * kLanes, H.slot_path.data(),
                          sizeof(long long) * H.slot_path.size(), cudaMemcpyHostToDevice, s));
    }
    b->views.resize(n);
    std::vector<std::vector<float>> dn_host(n);
    std::vector<std::vector<double>> dc_host(n);
    std::vector<std::vector<float>> cap_host(n);
    for (int i = 0; i < n; ++i) {
        const int j = lay_of[i];
        const te::HostLayout& H = hl[j];
        const te::BatchInst& I = b->inst[i];
        const size_t nd = (size_t)H.nblocks * b->dpb;
        // this instance's demands and capacities in the shared layout's order
        dn_host[i].assign(nd, 0.f);
        dc_host[i].assign(nd, 0.0);
        for (size_t d = 0; d < nd; ++d) {
            const int c = H.demand_of[d];
            if (c < 0) continue;
            dn_host[i][d] = (float)(demands[i][c] / b->scale[i]);
            dc_host[i][d] = demands[i][c];
        }
        cap_host[i].resize(E);
        for (int e = 0; e < E; ++e) cap_host[i][e] = (float)(capacities[i][e] / b->scale[i]);
        A(cudaMemcpyAsync(b->Dn + I.dslot0, dn_host[i].data(), sizeof(float) * nd, cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->Dc + I.dslot0, dc_host[i].data(), sizeof(double) * nd, cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->cap + (size_t)i * E, cap_host[i].data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->ne + (size_t)i * E, H.ne_f.data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
        A(cudaMemcpyAsync(b->inv + (size_t)i * E, H.inv_ne.data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
        // the instance's view of the concatenated arrays (instance-local indices)
        te::Layout& V = b->views[i];
        V.E = E;
        V.K = H.K;
        V.P = H.P;
        V.nnz = H.nnz;
        V.nblocks = H.nblocks;
        V.dpb = b->dpb;
        V.nslots = H.nslots;
        V.nrows = H.nrows;
        V.id_bytes = 2;
        V.kmax = H.kmax;
        V.G = G;
        V.kl = H.kl;
        V.max_block_rows = H.max_block_rows;
        V.ids = b->ids + (size_t)lrow0[j] * kLanes;
        V.rowoff = b->rowoff + lro[j];
        V.slotbase = b->slotbase + lso[j];
        V.blkmeta = b->blkmeta + lmeta0[j];
        V.hops = b->hops + (size_t)lmeta0[j] * kLanes;
        V.Dn = b->Dn + I.dslot0;
        V.np = b->np + (size_t)lmeta0[j] * b->dpb;
        V.demand_of = b->demand_of + (size_t)lmeta0[j] * b->dpb;
        V.slot_path = b->slot_path + (size_t)lslot0[j] * kLanes;
        V.cap_n = b->cap + (size_t)i * E;
        V.ne_f = b->ne + (size_t)i * E;
        V.inv_ne = b->inv + (size_t)i * E;
        b->bytes_per_iter += (long long)(sizeof(uint16_t) * H.ids.size()) + 8LL * H.nslots * kLanes +
                             12LL * (long long)nd + (long long)sizeof(te::BlockMeta) * H.nblocks;
    }
    A(cudaStreamSynchronize(s));  // the host staging vectors go out of scope below
    if (ce != cudaSuccess) {
        b->err = std::string("copy to device failed: ") + cudaGetErrorString(ce);
        return bail(TE_ECUDA);
    }
    b->hsc.resize(n);
    const te_status rs = te_batch_reset(b);
    if (rs != TE_OK) return bail(rs);
    *out = b;
    return TE_OK;
}

namespace {

te::BatchArgs batch_args(te_batch* b, long long iters) {
    te::BatchArgs a{};
    a.inst = b->d_inst;
    a.ninst = b->n;
    a.E = b->E;
    a.dpb = b->dpb;
    a.ids = b->ids;
    a.blkmeta = b->blkmeta;
    a.hops = b->hops;
    a.Dn = b->Dn;
    a.lam = b->lam;
    a.blkres = b->blkres;
    a.x = b->x;
    a.xstride = b->total_slots * kLanes;
    a.u = b->u;
    a.w = b->w;
    a.cap_n = b->cap;
    a.ne_f = b->ne;
    a.inv_ne = b->inv;
    a.sc = b->sc;
    a.o = b->o;
    a.max_iters = iters;
    a.timeout_ns = b->timeout_ns;
    a.status = b->status;
    a.next = b->next;
    return a;
}

// One launch over every instance for up to iters iterations each, in shape
// (W, ctas per SM); not captured.
cudaError_t batch_launch(te_batch* b, long long iters, int W, int ctas) {
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemsetAsync(b->next, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    b->launches += 1;
    return te::launch_batch(b->G, W, batch_args(b, iters), ctas, b->nsm, s);
}

// The instances in one cooperative launch of the iteration kernel, `group`
// CTAs each, for up to iters iterations each.
cudaError_t grouped_launch(te_batch* b, long long iters) {
    cudaStream_t s = b->stream;
    const int n = b->n, E = b->E, g = b->group;
    b->h_args.resize(n);
    for (int i = 0; i < n; ++i) {
        te::IterArgs a{};
        a.L = b->views[i];
        a.o = b->o;
        a.x = b->x + (size_t)b->inst[i].slot0 * kLanes;
        a.xstride = b->total_slots * kLanes;
        a.u = b->u + (size_t)i * E;
        a.w = b->w + (size_t)i * E;
        a.u_next = b->u_next + (size_t)i * E;
        a.w_next = b->w_next + (size_t)i * E;
        a.loads = b->gloads + (size_t)i * g * E;
        a.part = b->gpart + (size_t)i * 2 * g * te::kPartWidth;
        a.barrier = b->gbar + i;
        a.status = b->status;
        a.sc = b->sc + i;
        a.trace = nullptr;
        a.trace_cap = 0;
        a.lam = b->lam + b->inst[i].dslot0;
        a.max_iters = iters;
        a.timeout_ns = b->timeout_ns;
        b->h_args[i] = a;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_args, b->h_args.data(), sizeof(te::IterArgs) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->gbar, 0, sizeof(unsigned) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    b->launches += 1;
    return te::launch_iter_grouped(b->d_args, n, g, b->G, E, s);
}

}  // namespace

extern "C" te_status te_batch_solve(te_batch* b, int64_t max_iters, te_solve_result* results) {
    if (!b || max_iters < 0) return TE_EINVAL;
    cudaStream_t s = b->stream;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    const std::vector<te::Scalars> before = b->hsc;
    long long left = max_iters;
    if (b->group > 0) {
        // the host copy of h_args stays alive until the stream synchronises below
        if (left > 0) A(grouped_launch(b, left));
        left = 0;
    }
    // first call: time each CTA shape on the batch's own first iterations
    if (b->shape_w == 0 && left > 0) {
        float best = 0.f;
        for (int W : te::kShapes) {
            int occ = 0;
            if (te::batch_occupancy(b->G, W, b->E, &occ) != cudaSuccess || occ < 1) {
                cudaGetLastError();
                continue;
            }
            for (int ctas = 1; ctas <= std::min(occ, 2); ++ctas) {
                const long long chunk = std::min<long long>(left, 5);
                if (chunk <= 0) break;
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, s);
                A(batch_launch(b, chunk, W, ctas));
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                left -= chunk;
                b->shape_ms.push_back(ms / (float)chunk);
                if (b->shape_w == 0 || ms / chunk < best) {
                    best = ms / chunk;
                    b->shape_w = W;
                    b->shape_ctas = ctas;
                }
                if (ce != cudaSuccess) return b->cuda(ce, "te_batch_solve");
            }
        }
        if (b->shape_w == 0) return b->fail(TE_EUNSUPPORTED, "no CTA shape of the batch kernel fits an SM");
    }
    if (left > 0) {
        auto g = b->graphs.find(left);
        if (g == b->graphs.end()) {
            cudaGraph_t graph;
            A(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            A(batch_launch(b, left, b->shape_w, b->shape_ctas));
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            A(ee);
            if (ce != cudaSuccess) return b->cuda(ce, "te_batch_solve (graph capture)");
            cudaGraphExec_t exec;
            A(cudaGraphInstantiate(&exec, graph, 0));
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return b->cuda(ce, "te_batch_solve (graph instantiate)");
            g = b->graphs.emplace(left, exec).first;
        } else {
            b->launches += 1;
        }
        A(cudaGraphLaunch(g->second, s));
    }
    int status = 0;
    A(cudaMemcpyAsync(&status, b->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    A(cudaMemcpyAsync(b->hsc.data(), b->sc, sizeof(te::Scalars) * b->n, cudaMemcpyDeviceToHost, s));
    A(cudaStreamSynchronize(s));
    if (ce != cudaSuccess) return b->cuda(ce, "te_batch_solve");
    if (results) {
        for (int i = 0; i < b->n; ++i) {
            const te::Scalars& c = b->hsc[i];
            results[i].iters = c.iter_total - before[i].iter_total;
            results[i].total_iters = c.iter_total;
            results[i].r = c.r;
            results[i].s = c.s;
            results[i].beta = c.beta;
            results[i].alpha = c.alpha;
            results[i].converged = c.converged;
            results[i].stop_reason = c.stop_reason;
        }
    }
    if (status == te::kStatusTimeout) return b->fail(TE_ETIMEOUT, "a kernel wait ran past its time limit");
    if (status == te::kStatusNumeric) return b->fail(TE_ENUMERIC, "a residual is not finite");
    return TE_OK;
}

extern "C" te_status te_batch_allocation(te_batch* b, int32_t i, float* x_out, int32_t project, int32_t out_is_device) {
    if (!b || !x_out || i < 0 || i >= b->n || project < TE_PROJECT_NONE || project > TE_PROJECT_SCALE) return TE_EINVAL;
    cudaStream_t s = b->stream;
    const te::Layout& V = b->views[i];
    const size_t ns = (size_t)V.nslots * kLanes;
    const float* src = b->x + (size_t)b->hsc[i].xbuf * b->total_slots * kLanes + (size_t)b->inst[i].slot0 * kLanes;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    if (project != TE_PROJECT_NONE) {
        A(cudaMemcpyAsync(b->xtmp, src, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
        if (project == TE_PROJECT_ALG2) {
            int np_ = 0;
            A(te::launch_project(V, b->xtmp, b->hsc[i].alpha, b->scale[i], b->ps, s, &np_));
            b->launches += np_;
        } else {
            A(te::launch_project_scale(V, b->xtmp, b->ps, s));
            b->launches += te::kProjectScaleLaunches;
        }
        src = b->xtmp;
    }
    float* dst = out_is_device ? x_out : b->user;
    A(te::launch_to_user(V, src, dst, (float)b->scale[i], s));
    b->launches += 1;
    if (!out_is_device) A(cudaMemcpyAsync(x_out, b->user, sizeof(float) * (size_t)V.P, cudaMemcpyDeviceToHost, s));
    A(cudaStreamSynchronize(s));
    return b->cuda(ce, "te_batch_allocation");
}

extern "C" te_status te_batch_info(const te_batch* b, te_batch_info_t* info) {
    if (!b || !info) return TE_EINVAL;
    info->n_instances = b->n;
    long long P = 0;
    for (long long p : b->P) P += p;
    info->n_paths = P;
    info->id_rows = b->total_rows;
    info->bytes_per_iter = b->bytes_per_iter;
    info->device_bytes = b->device_bytes;
    info->kernel_launches = b->launches;
    info->warps_per_cta = b->group > 0 ? te::kIterWarps : b->shape_w;
    info->ctas_per_sm = b->group > 0 ? 1 : b->shape_ctas;
    info->lanes_per_demand = b->G;
    info->ctas_per_instance = b->group;
    return TE_OK;
}

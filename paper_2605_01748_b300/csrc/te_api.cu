// Host side of the C-ABI (include/te.h): input validation, the sliced device
// layout, device memory, kernel launches and error reporting.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "te.h"
#include "te_layout.h"
#include "te_literal.h"
#include "te_internal.cuh"
#include "te_proj.h"
#include "te_adjoint.h"

using te::kLanes;

namespace {

thread_local std::string g_create_error;

constexpr long long kTraceCap = 1 << 16;
constexpr long long kItersPerLaunch = 1LL << 22;  // two barriers per iteration: counter below 2^32

// p_out[e] = pscale * u[e]
__global__ void k_prices(int E, const float* u, double pscale, double* p) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) p[e] = pscale * (double)u[e];
}

// flags demands that are not finite and positive
__global__ void k_check_demands(int K, const double* D, int* bad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < K && !(D[c] > 0.0 && D[c] < INFINITY)) atomicOr(bad, 1);
}

// new demands into demand-slot order: normalised FP32 for the iteration,
// caller units FP64 for the gap
__global__ void k_set_demands(long long nd, const int* demand_of, const double* D, double inv_scale, float* Dn,
                              double* Dc) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nd) return;
    const int c = demand_of[i];
    if (c < 0) return;
    Dn[i] = (float)(D[c] * inv_scale);
    Dc[i] = D[c];
}

__global__ void k_check_capacities(int E, const double* C, int* bad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E && !(C[e] >= 0.0 && C[e] < INFINITY)) atomicOr(bad, 1);
}

// new capacities, normalised FP32
__global__ void k_set_capacities(int E, const double* C, double inv_scale, float* cap_n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) cap_n[e] = (float)(C[e] * inv_scale);
}

}  // namespace

namespace te {
cudaError_t launch_prices(int E, const float* u, double pscale, double* p_out, cudaStream_t st) {
    k_prices<<<(E + 255) / 256, 256, 0, st>>>(E, u, pscale, p_out);
    return cudaGetLastError();
}
}  // namespace te

struct te_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    te::Options o{};
    double beta0 = 1.0;
    long long timeout_ns = 2000000000LL;
    te::Layout L{};
    double scale = 1.0;
    int grid = 0;
    long long bytes_per_iter = 0;
    long long device_bytes = 0;
    // owned device buffers
    std::vector<void*> owned;
    float* x = nullptr;       // [2][nslots*32]
    float* u = nullptr;       // [E]
    float* w = nullptr;       // [E]
    float* u_next = nullptr;  // [E]
    float* w_next = nullptr;  // [E]
    uint2* loads = nullptr;   // [grid*E] per-CTA partial loads
    bool wide = false;        // per-edge arrays of the iteration kernel in global memory
    unsigned long long* hist64 = nullptr;  // [grid*(E+1)] wide mode: per-CTA load histograms
    float* wpriv = nullptr;                // [grid*(E+1)] wide mode: per-CTA gather weights
    double* part = nullptr;   // [2*grid*kPartWidth]
    unsigned* barrier = nullptr;
    int* status = nullptr;
    te::Scalars* sc = nullptr;
    double* trace = nullptr;  // [kTraceCap*5]
    double* Dc = nullptr;     // [nblocks*dpb] caller-unit demands
    float* xtmp = nullptr;    // [nslots*32]
    float* user = nullptr;    // [P]
    double* gacc = nullptr;   // [3]
    double* gslots = nullptr; // [2*gap_slot_count] per-CTA partials of the gap
    double* pbuf = nullptr;   // [E]
    double* dstage = nullptr; // [K] staging of new demands
    double* cstage = nullptr; // [E] staging of new capacities
    float* cap_n = nullptr;   // [E] normalised capacities (the layout's copy)
    int* flag = nullptr;      // [1]
    float* lam = nullptr;     // [nblocks*dpb] warm-start multipliers
    float* Dn = nullptr;      // mutable view of L.Dn
    long long launches = 0;   // kernels launched through this handle
    te::ProjScratch ps{};
    te::Scalars hsc{};        // host mirror of the scalars
    std::string err;

    te_status fail(te_status s, const std::string& m) {
        err = m;
        return s;
    }
    te_status cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return TE_OK;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return TE_ECUDA;
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) {
            owned.push_back(q);
            device_bytes += (long long)bytes;
        }
        *p = (T*)q;
        return e;
    }
};

extern "C" {

void te_default_options(te_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->alpha_target = INFINITY;
    o->alpha_start = 0.0;
    o->alpha_step = 1.0;
    o->alpha_max = 32.0;
    o->gamma = 1e-3;
    o->A = 10.0;
    o->C = 2.0;
    o->beta0 = 0.0;       // automatic (see te.h)
    o->balance_floor = 1e-6;
    o->gamma_max = 0.0;
    o->beta_max = 0.0;
    o->adapt_beta = 1;
    o->continuation = 1;
    o->scale_mode = 1;    // geometric mean of the demands
    o->wait_timeout_ms = 0;
    o->test_withhold_cta = 0;
    o->deterministic = 1;
    o->precision = TE_PRECISION_FP32;
    o->edge_mode = TE_EDGES_AUTO;
    o->cuda_stream = nullptr;
}

const char* te_last_error(const te_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void te_destroy(te_handle* h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->owned) cudaFree(p);
    if (h->ps.vlist) cudaFree(h->ps.vlist);
    cudaSetDevice(cur);
    delete h;
}

}  // extern "C"

namespace {

std::string fmt(const char* f, long long a, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

// Checks the instance; returns an empty string when valid.
std::string validate(const te_topology* topo, const te_paths* P, const double* D, const double* C) {
    if (!topo || !P || !D || !C) return "null argument";
    const int E = topo->n_edges;
    if (E <= 0) return "n_edges must be positive";
    if (E >= 0x7ffffffe) return "n_edges too large";
    if (P->n_demands <= 0) return "n_demands must be positive";
    if (P->n_paths < P->n_demands) return "fewer paths than demands";
    if (P->nnz < P->n_paths) return "fewer incidences than paths";
    if (!P->demand_path_off || !P->path_edge_off || !P->path_edges) return "null path arrays";
    const int K = P->n_demands;
    if (P->demand_path_off[0] != 0 || P->demand_path_off[K] != P->n_paths)
        return "demand_path_off must start at 0 and end at n_paths";
    if (P->path_edge_off[0] != 0 || P->path_edge_off[P->n_paths] != P->nnz)
        return "path_edge_off must start at 0 and end at nnz";
    for (int c = 0; c < K; ++c) {
        const long long k = P->demand_path_off[c + 1] - P->demand_path_off[c];
        if (k < 1) return fmt("demand %lld has no path", c);
        if (k > te::kMaxPaths) return fmt("demand %lld has %lld paths (limit 32)", c, k);
        if (!(D[c] > 0.0) || !isfinite(D[c])) return fmt("demand %lld is not finite and positive", c);
    }
    for (long long r = 0; r < P->n_paths; ++r) {
        const long long n = P->path_edge_off[r + 1] - P->path_edge_off[r];
        if (n < 1) return fmt("path %lld is empty", r);
        if (n > te::kMaxHops) return fmt("path %lld has %lld edges (limit 255)", r, n);
    }
    std::vector<char> used(E, 0);
    for (long long i = 0; i < P->nnz; ++i) {
        const int e = P->path_edges[i];
        if (e < 0 || e >= E) return fmt("incidence %lld names edge %lld out of range", i, e);
        used[e] = 1;
    }
    for (int e = 0; e < E; ++e) {
        if (!isfinite(C[e]) || C[e] < 0.0) return fmt("capacity of edge %lld is not finite and >= 0", e);
        if (used[e] && !(C[e] > 0.0)) return fmt("edge %lld is on a path but has zero capacity", e);
    }
    if (topo->edge_src && topo->edge_dst) {
        const int N = topo->n_nodes;
        for (int e = 0; e < E; ++e)
            if (topo->edge_src[e] < 0 || topo->edge_src[e] >= N || topo->edge_dst[e] < 0 || topo->edge_dst[e] >= N)
                return fmt("edge %lld has an endpoint out of range", e);
        if (P->demand_src && P->demand_dst) {
            for (int c = 0; c < K; ++c) {
                for (long long r = P->demand_path_off[c]; r < P->demand_path_off[c + 1]; ++r) {
                    const long long i0 = P->path_edge_off[r], i1 = P->path_edge_off[r + 1];
                    if (topo->edge_src[P->path_edges[i0]] != P->demand_src[c] ||
                        topo->edge_dst[P->path_edges[i1 - 1]] != P->demand_dst[c])
                        return fmt("path %lld does not join its demand's endpoints", r);
                    for (long long i = i0; i + 1 < i1; ++i)
                        if (topo->edge_dst[P->path_edges[i]] != topo->edge_src[P->path_edges[i + 1]])
                            return fmt("path %lld is not a walk", r);
                }
            }
        }
    }
    return "";
}

}  // namespace

extern "C" te_status te_create(const te_topology* topo, const te_paths* P, const double* D, const double* C,
                               const te_options* opt_in, te_handle** out) {
    g_create_error.clear();
    if (!out) { g_create_error = "null output handle"; return TE_EINVAL; }
    *out = nullptr;
    {
        std::string v = validate(topo, P, D, C);
        if (!v.empty()) { g_create_error = v; return TE_EINVAL; }
    }
    te_options opt;
    if (opt_in) opt = *opt_in; else te_default_options(&opt);
    if (!(opt.gamma == opt.gamma) || !(opt.beta0 == opt.beta0) || !(opt.balance_floor >= 0.0) || !(opt.gamma_max == opt.gamma_max) || !(opt.beta_max >= 0.0) || !(opt.C > 1.0) || !(opt.A > 0.0) ||
        (opt.scale_mode < 0 || opt.scale_mode > 2) || (opt.deterministic != 0 && opt.deterministic != 1) ||
        (opt.edge_mode != TE_EDGES_AUTO && opt.edge_mode != TE_EDGES_GLOBAL) ||
        !(opt.alpha_step > 0.0) || opt.alpha_start < 0.0 || opt.alpha_target < 0.0 || opt.alpha_max < 0.0) {
        g_create_error = "invalid options";
        return TE_EINVAL;
    }
    if (opt.precision != TE_PRECISION_FP32) {
        g_create_error = "precision: only TE_PRECISION_FP32 is implemented";
        return TE_EUNSUPPORTED;
    }
    te_handle* h = new (std::nothrow) te_handle();
    if (!h) { g_create_error = "out of host memory"; return TE_ENOMEM; }
    auto bail = [&](te_status s) {
        g_create_error = h->err;
        te_destroy(h);
        return s;
    };
    cudaGetDevice(&h->device);
    h->stream = (cudaStream_t)opt.cuda_stream;
    h->o.alpha_target = opt.alpha_target;
    h->o.alpha_start = opt.alpha_start;
    h->o.alpha_step = opt.alpha_step;
    h->o.alpha_max = opt.alpha_max;
    h->o.gamma = opt.gamma;
    h->o.A = opt.A;
    h->o.C = opt.C;
    h->o.adapt_beta = opt.adapt_beta;
    h->o.continuation = opt.continuation;
    h->o.balance_floor = opt.balance_floor;
    h->o.gamma_max = opt.gamma_max;
    h->o.beta_cap = 1e30;
    h->o.deterministic = opt.deterministic;
    h->o.withhold_cta = opt.test_withhold_cta > 0 ? opt.test_withhold_cta - 1 : -1;
    h->beta0 = opt.beta0;
    if (opt.wait_timeout_ms > 0) h->timeout_ns = (long long)opt.wait_timeout_ms * 1000000LL;

    const int E = topo->n_edges;
    const int K = P->n_demands;
    const long long NP = P->n_paths;
    double scale = 0.0;
    if (opt.scale_mode == 1) {
        double lg = 0.0;
        for (int c = 0; c < K; ++c) lg += log(D[c]);
        scale = exp(lg / (double)K);
    } else if (opt.scale_mode == 2) {
        scale = 1.0;  // caller units
    } else {
        for (int e = 0; e < E; ++e) scale = std::max(scale, C[e]);
    }
    h->scale = scale;
    if (!(opt.beta0 > 0.0)) {
        // first push lambda/(beta n_r) at lambda = 1 equal to the mean initial rate
        double dsum = 0.0;
        for (int c = 0; c < K; ++c) dsum += D[c] / scale;
        const double xbar = dsum / (double)NP, nbar = (double)P->nnz / (double)NP;
        h->beta0 = 1.0 / (nbar * xbar);
    }

    // ---------------- sliced layout ----------------
    te::HostLayout hl;
    {
        const te_status ls = te::build_host_layout(topo, P, D, C, scale, 1, hl, 4);
        if (ls != TE_OK) { h->err = hl.err; return bail(ls); }
    }
    const int G = hl.G, DPB = hl.dpb, kl = hl.kl, kmax = hl.kmax, nblocks = hl.nblocks;
    const int max_block_rows = hl.max_block_rows;
    const long long nslots = hl.nslots, nrows = hl.nrows;
    const int id_bytes = hl.id_bytes;  // 4 above 65,534 edges (wide-edge mode only)
    const size_t n_ids = id_bytes == 4 ? hl.ids32.size() : hl.ids.size();
    const void* h_ids = id_bytes == 4 ? (const void*)hl.ids32.data() : (const void*)hl.ids.data();
    const size_t ND = (size_t)nblocks * DPB;  // demand slots

    // ---------------- persistent grid ----------------
    int bps = 0, nsm = 0;
    te_status st;
    if ((st = h->cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device), "device query")))
        return bail(st);
    // per-edge arrays of the iteration kernel in shared memory when they fit,
    // else (or when asked) in global memory
    h->wide = opt.edge_mode == TE_EDGES_GLOBAL || id_bytes == 4 ||
              te::iter_smem_bytes(E, nsm, opt.deterministic != 0) > 227 * 1024;
    if (h->wide && opt.deterministic == 0) {
        h->err = fmt("n_edges = %lld: the per-edge arrays exceed a CTA's shared memory (about 10770 edges) or "
                     "edge_mode asks for global memory, which needs deterministic = 1", E);
        return bail(TE_EUNSUPPORTED);
    }
    if (h->wide && te::iter_smem_bytes_wide(E, nsm, id_bytes) > 227 * 1024 - 1024) {
        // the staging buffers and each CTA's slice of the prices must fit
        h->err = fmt("n_edges = %lld: the iteration kernel's price slices exceed shared memory (at most "
                     "about 490,000 edges)", E);
        return bail(TE_EUNSUPPORTED);
    }
    if (h->wide) {
        if ((st = h->cuda(te::iter_occupancy_wide(G, id_bytes, E, nsm, &bps), "occupancy query"))) return bail(st);
    } else if ((st = h->cuda(te::iter_occupancy(G, opt.deterministic != 0, E, nsm, &bps), "occupancy query"))) {
        return bail(st);
    }
    if (bps < 1) { h->err = "iteration kernel does not fit on an SM"; return bail(TE_EUNSUPPORTED); }
    h->grid = nsm * bps;

    // ---------------- device memory ----------------
    void* d_ids;
    unsigned* d_rowoff;
    int *d_slotbase, *d_demand_of;
    te::BlockMeta* d_blkmeta;
    unsigned* d_hops;
    float *d_Dn, *d_cap, *d_ne, *d_inv;
    unsigned char* d_np;
    long long* d_slot_path;
    const size_t ns = (size_t)nslots * kLanes;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    A(h->alloc(&d_ids, (size_t)id_bytes * n_ids));
    A(h->alloc(&d_rowoff, sizeof(unsigned) * hl.rowoff.size()));
    A(h->alloc(&d_slotbase, sizeof(int) * hl.slotbase.size()));
    A(h->alloc(&d_demand_of, sizeof(int) * ND));
    A(h->alloc(&d_blkmeta, sizeof(te::BlockMeta) * (size_t)nblocks));
    A(h->alloc(&d_hops, sizeof(unsigned) * hl.hops.size()));
    A(h->alloc(&d_Dn, sizeof(float) * ND));
    A(h->alloc(&h->Dc, sizeof(double) * ND));
    A(h->alloc(&d_np, ND));
    A(h->alloc(&d_slot_path, sizeof(long long) * ns));
    A(h->alloc(&d_cap, sizeof(float) * E));
    A(h->alloc(&d_ne, sizeof(float) * E));
    A(h->alloc(&d_inv, sizeof(float) * E));
    A(h->alloc(&h->x, sizeof(float) * 2 * ns));
    A(h->alloc(&h->u, sizeof(float) * E));
    A(h->alloc(&h->w, sizeof(float) * E));
    A(h->alloc(&h->u_next, sizeof(float) * E));
    A(h->alloc(&h->w_next, sizeof(float) * E));
    if (h->wide) {
        A(h->alloc(&h->hist64, sizeof(unsigned long long) * (size_t)h->grid * (size_t)(E + 1)));
        A(h->alloc(&h->wpriv, sizeof(float) * (size_t)h->grid * (size_t)(E + 1)));
    } else {
        A(h->alloc(&h->loads, sizeof(uint2) * (size_t)h->grid * (size_t)E));
    }
    A(h->alloc(&h->part, sizeof(double) * 2 * te::kPartWidth * (size_t)h->grid));
    A(h->alloc(&h->barrier, sizeof(unsigned)));
    A(h->alloc(&h->status, sizeof(int)));
    A(h->alloc(&h->sc, sizeof(te::Scalars)));
    A(h->alloc(&h->trace, sizeof(double) * te::kTraceWidth * kTraceCap));
    A(h->alloc(&h->xtmp, sizeof(float) * ns));
    A(h->alloc(&h->user, sizeof(float) * (size_t)NP));
    A(h->alloc(&h->gacc, sizeof(double) * 4));
    {
        te::Layout lg{};
        lg.nblocks = nblocks;
        lg.dpb = DPB;
        A(h->alloc(&h->gslots, sizeof(double) * 2 * te::gap_slot_count(lg)));
    }
    A(h->alloc(&h->pbuf, sizeof(double) * E));
    A(h->alloc(&h->dstage, sizeof(double) * K));
    A(h->alloc(&h->cstage, sizeof(double) * E));
    A(h->alloc(&h->flag, sizeof(int)));
    A(h->alloc(&h->lam, sizeof(float) * ND));
    A(h->alloc(&h->ps.S, sizeof(double) * ND));
    A(h->alloc(&h->ps.loads, sizeof(unsigned long long) * E));
    A(h->alloc(&h->ps.viol, (size_t)E));
    A(h->alloc(&h->ps.vidx, sizeof(int) * E));
    A(h->alloc(&h->ps.nviol, sizeof(int)));
    A(h->alloc(&h->ps.hist, sizeof(unsigned long long) * 256 * (size_t)E));
    A(h->alloc(&h->ps.prefix, sizeof(unsigned long long) * E));
    A(h->alloc(&h->ps.rem, sizeof(double) * E));
    A(h->alloc(&h->ps.Cp, ns));
    A(h->alloc(&h->ps.score, sizeof(double) * (ND + 256)));
    A(h->alloc(&h->ps.vtotal, 3 * sizeof(unsigned long long)));
    if (ce != cudaSuccess) {
        h->err = std::string("device allocation failed: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return bail(ce == cudaErrorMemoryAllocation ? TE_ENOMEM : TE_ECUDA);
    }
    cudaStream_t s = h->stream;
    A(cudaMemcpyAsync(d_ids, h_ids, (size_t)id_bytes * n_ids, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_rowoff, hl.rowoff.data(), sizeof(unsigned) * hl.rowoff.size(), cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_slotbase, hl.slotbase.data(), sizeof(int) * hl.slotbase.size(), cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_demand_of, hl.demand_of.data(), sizeof(int) * ND, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_blkmeta, hl.blkmeta.data(), sizeof(te::BlockMeta) * (size_t)nblocks, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_hops, hl.hops.data(), sizeof(unsigned) * hl.hops.size(), cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_Dn, hl.Dn.data(), sizeof(float) * ND, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(h->Dc, hl.Dc.data(), sizeof(double) * ND, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_np, hl.np.data(), ND, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_slot_path, hl.slot_path.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_cap, hl.cap_n.data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_ne, hl.ne_f.data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
    A(cudaMemcpyAsync(d_inv, hl.inv_ne.data(), sizeof(float) * E, cudaMemcpyHostToDevice, s));
    if (ce != cudaSuccess) {
        h->err = std::string("copy to device failed: ") + cudaGetErrorString(ce);
        return bail(TE_ECUDA);
    }
    te::Layout& L = h->L;
    L.E = E;
    L.K = K;
    L.P = NP;
    L.nnz = P->nnz;
    L.nblocks = nblocks;
    L.dpb = DPB;
    L.max_block_rows = max_block_rows;
    L.blkmeta = d_blkmeta;
    L.hops = d_hops;
    L.nslots = nslots;
    L.nrows = nrows;
    L.id_bytes = id_bytes;
    L.kmax = kmax;
    L.G = G;
    L.kl = kl;
    L.ids = d_ids;
    L.rowoff = d_rowoff;
    L.slotbase = d_slotbase;
    L.Dn = d_Dn;
    h->Dn = d_Dn;
    L.np = d_np;
    L.demand_of = d_demand_of;
    L.slot_path = d_slot_path;
    L.cap_n = d_cap;
    h->cap_n = d_cap;
    L.ne_f = d_ne;
    L.inv_ne = d_inv;
    // algorithmic traffic of one iteration: the edge ids once, the rates read
    // and written, per demand its value and its multiplier read and written,
    // per block its metadata record and its lanes' hop counts
    h->bytes_per_iter = (long long)((size_t)id_bytes * n_ids) + 2LL * (long long)sizeof(float) * (long long)ns +
                        3LL * (long long)sizeof(float) * (long long)ND +
                        (long long)sizeof(te::BlockMeta) * (long long)nblocks +
                        (long long)sizeof(unsigned) * (long long)hl.hops.size();
    if (opt.beta_max > 0.0) h->o.beta_cap = opt.beta_max * h->beta0;
    te_status rs = te_reset(h);
    if (rs != TE_OK) return bail(rs);
    *out = h;
    return TE_OK;
}

extern "C" te_status te_reset(te_handle* h) {
    if (!h) return TE_EINVAL;
    cudaStream_t s = h->stream;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    A(te::launch_init_x(h->L, h->x, s));
    h->launches += 1;
    A(cudaMemsetAsync(h->u, 0, sizeof(float) * h->L.E, s));
    A(cudaMemsetAsync(h->w, 0, sizeof(float) * h->L.E, s));
    A(cudaMemsetAsync(h->lam, 0, sizeof(float) * (size_t)h->L.nblocks * h->L.dpb, s));
    te::Scalars sc{};
    sc.beta = h->beta0;
    sc.alpha = (isfinite(h->o.alpha_target) && h->o.alpha_start > h->o.alpha_target) ? h->o.alpha_target
                                                                                     : h->o.alpha_start;
    h->hsc = sc;
    A(cudaMemcpyAsync(h->sc, &h->hsc, sizeof(sc), cudaMemcpyHostToDevice, s));
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_reset");
}

extern "C" te_status te_literal_run(const te_topology* topo, const te_paths* paths, const double* demands,
                                   const double* capacities, double alpha, double beta, int64_t iters,
                                   double* x_out, void* cuda_stream) {
    g_create_error.clear();
    if (!x_out || !(alpha >= 0.0) || !isfinite(alpha) || !(beta > 0.0) || !isfinite(beta) || iters < 0) {
        g_create_error = "te_literal_run: null output, alpha < 0, beta <= 0 or iters < 0";
        return TE_EINVAL;
    }
    const std::string v = validate(topo, paths, demands, capacities);
    if (!v.empty()) {
        g_create_error = v;
        return TE_EINVAL;
    }
    if (paths->nnz > 0x7fffffffLL) {  // the incidence lists hold 32-bit indices
        g_create_error = "te_literal_run: more than 2^31 - 1 path-edge incidences";
        return TE_EUNSUPPORTED;
    }
    std::string err;
    const te_status st = te::literal_run(paths, topo->n_edges, demands, capacities, alpha, beta, iters, x_out,
                                         static_cast<cudaStream_t>(cuda_stream), err);
    if (st != TE_OK) g_create_error = err;
    return st;
}

extern "C" te_status te_solve(te_handle* h, int64_t max_iters, double tol, te_solve_result* out) {
    if (!h) return TE_EINVAL;
    if (max_iters < 0) return h->fail(TE_EINVAL, "max_iters must be >= 0");
    if (tol != tol) return h->fail(TE_EINVAL, "tol is NaN");
    const double gamma = tol >= 0.0 ? tol : h->o.gamma;
    cudaStream_t s = h->stream;
    long long done = 0;
    te_status rc = TE_OK;
    int converged = 0, reason = 0;
    while (done < max_iters || (max_iters == 0 && done == 0)) {
        const long long chunk = std::min<long long>(max_iters - done, kItersPerLaunch);
        if (chunk <= 0) break;
        cudaError_t ce = cudaSuccess;
        auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
        A(cudaMemsetAsync(h->barrier, 0, sizeof(unsigned), s));
        A(cudaMemsetAsync(h->status, 0, sizeof(int), s));
        te::IterArgs a{};
        a.L = h->L;
        a.o = h->o;
        a.o.gamma = gamma;
        a.x = h->x;
        a.u = h->u;
        a.w = h->w;
        a.loads = h->loads;
        a.hist64 = h->hist64;
        a.wpriv = h->wpriv;
        a.part = h->part;
        a.barrier = h->barrier;
        a.status = h->status;
        a.sc = h->sc;
        a.trace = h->trace;
        a.trace_cap = kTraceCap;
        a.lam = h->lam;
        a.u_next = h->u_next;
        a.w_next = h->w_next;
        a.max_iters = chunk;
        a.timeout_ns = h->timeout_ns;
        A(te::launch_iter(a, h->grid, s));
        h->launches += 1;
        int status = 0;
        A(cudaMemcpyAsync(&h->hsc, h->sc, sizeof(te::Scalars), cudaMemcpyDeviceToHost, s));
        A(cudaMemcpyAsync(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        A(cudaStreamSynchronize(s));
        if (ce != cudaSuccess) return h->cuda(ce, "te_solve");
        done += h->hsc.iters_run;
        if (status == te::kStatusTimeout) {
            rc = h->fail(TE_ETIMEOUT, "a grid-wide wait exceeded its time limit; state of the last completed "
                                      "iteration kept");
            break;
        }
        if (status == te::kStatusNumeric) {
            rc = h->fail(TE_ENUMERIC, "a residual became NaN or Inf");
            break;
        }
        if (h->hsc.converged) {
            converged = 1;
            reason = h->hsc.stop_reason;
            break;
        }
        if (h->hsc.iters_run < chunk) break;
    }
    if (out) {
        out->iters = done;
        out->total_iters = h->hsc.iter_total;
        out->r = h->hsc.r;
        out->s = h->hsc.s;
        out->beta = h->hsc.beta;
        out->alpha = h->hsc.alpha;
        out->converged = converged;
        out->stop_reason = reason;
    }
    return rc;
}

extern "C" te_status te_allocation(te_handle* h, float* x_out, int32_t project, int32_t out_is_device) {
    if (!h || !x_out || project < TE_PROJECT_NONE || project > TE_PROJECT_SCALE) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const size_t ns = (size_t)h->L.nslots * kLanes;
    const float* src = h->x + (size_t)h->hsc.xbuf * ns;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    if (project != TE_PROJECT_NONE) {
        A(cudaMemcpyAsync(h->xtmp, src, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
        if (project == TE_PROJECT_ALG2) {
            int np_ = 0;
            A(te::launch_project(h->L, h->xtmp, h->hsc.alpha, h->scale, h->ps, s, &np_));
            h->launches += np_;
        } else {
            A(te::launch_project_scale(h->L, h->xtmp, h->ps, s));
            h->launches += te::kProjectScaleLaunches;
        }
        src = h->xtmp;
    }
    float* dst = out_is_device ? x_out : h->user;
    A(te::launch_to_user(h->L, src, dst, (float)h->scale, s));
    h->launches += 1;
    if (!out_is_device)
        A(cudaMemcpyAsync(x_out, h->user, sizeof(float) * (size_t)h->L.P, cudaMemcpyDeviceToHost, s));
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_allocation");
}

extern "C" te_status te_gap_projected(te_handle* h, int32_t project, double* gap_out, double* primal_out,
                                      double* dual_out) {
    if (!h || (project != TE_PROJECT_ALG2 && project != TE_PROJECT_SCALE)) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const size_t ns = (size_t)h->L.nslots * kLanes;
    const float* src = h->x + (size_t)h->hsc.xbuf * ns;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    A(cudaMemcpyAsync(h->xtmp, src, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
    if (project == TE_PROJECT_ALG2) {
        int np_ = 0;
        A(te::launch_project(h->L, h->xtmp, h->hsc.alpha, h->scale, h->ps, s, &np_));
        h->launches += np_;
    } else {
        A(te::launch_project_scale(h->L, h->xtmp, h->ps, s));
        h->launches += te::kProjectScaleLaunches;
    }
    A(te::launch_gap_impl(h->L, h->xtmp, h->u, h->hsc.beta, h->hsc.alpha, h->scale, h->Dc, h->gacc, h->gslots, s));
    h->launches += te::kGapLaunches;
    double acc[4] = {0, 0, 0, 0};
    A(cudaMemcpyAsync(acc, h->gacc, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    A(cudaStreamSynchronize(s));
    if (ce != cudaSuccess) return h->cuda(ce, "te_gap");
    const double primal = acc[0], dual = acc[1] + acc[2];
    if (gap_out) *gap_out = dual - primal;
    if (primal_out) *primal_out = primal;
    if (dual_out) *dual_out = dual;
    return TE_OK;
}

extern "C" te_status te_gap(te_handle* h, double* gap_out, double* primal_out, double* dual_out) {
    return te_gap_projected(h, TE_PROJECT_ALG2, gap_out, primal_out, dual_out);
}

extern "C" te_status te_prices(te_handle* h, double* p_out, int32_t out_is_device) {
    if (!h || !p_out) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const double pscale = h->hsc.beta * pow(h->scale, -h->hsc.alpha);
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    double* dst = out_is_device ? p_out : h->pbuf;
    A(te::launch_prices(h->L.E, h->u, pscale, dst, s));
    h->launches += 1;
    if (!out_is_device) A(cudaMemcpyAsync(p_out, h->pbuf, sizeof(double) * h->L.E, cudaMemcpyDeviceToHost, s));
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_prices");
}

extern "C" te_status te_set_warm_start(te_handle* h, const float* x0, int32_t in_is_device, int32_t keep_duals) {
    if (!h || !x0) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const size_t ns = (size_t)h->L.nslots * kLanes;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    const float* src = x0;
    if (!in_is_device) {
        A(cudaMemcpyAsync(h->user, x0, sizeof(float) * (size_t)h->L.P, cudaMemcpyHostToDevice, s));
        src = h->user;
    }
    if (!keep_duals) {
        te_status r = te_reset(h);
        if (r != TE_OK) return r;
    }
    A(te::launch_from_user(h->L, src, h->x + (size_t)h->hsc.xbuf * ns, (float)(1.0 / h->scale), s));
    h->launches += 1;
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_set_warm_start");
}

extern "C" te_status te_trace(te_handle* h, double* out, int64_t max_rows, int64_t* rows) {
    if (!h || (!out && max_rows > 0) || max_rows < 0) return TE_EINVAL;
    const long long total = h->hsc.iter_total;
    const long long avail = std::min<long long>(total, kTraceCap);
    const long long n = std::min<long long>(avail, max_rows);
    std::vector<double> ring((size_t)kTraceCap * te::kTraceWidth);
    cudaError_t ce = cudaMemcpyAsync(ring.data(), h->trace, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost,
                                     h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return h->cuda(ce, "te_trace");
    // oldest row first
    const long long first = total - avail;
    for (long long i = 0; i < n; ++i) {
        const long long it = first + i;
        memcpy(out + i * te::kTraceWidth, ring.data() + (size_t)(it % kTraceCap) * te::kTraceWidth,
               sizeof(double) * te::kTraceWidth);
    }
    if (rows) *rows = n;
    return TE_OK;
}

extern "C" te_status te_layout(const te_handle* h, te_layout_info* info) {
    if (!h || !info) return TE_EINVAL;
    info->n_demands = h->L.K;
    info->n_paths = h->L.P;
    info->nnz = h->L.nnz;
    info->id_rows = h->L.nrows;
    info->slots = h->L.nslots;
    info->id_bytes = h->L.id_bytes;
    info->grid = h->grid;
    info->bytes_per_iter = h->bytes_per_iter;
    info->device_bytes = h->device_bytes;
    info->kernel_launches = h->launches;
    info->edges_global = h->wide ? 1 : 0;
    info->reserved = 0;
    return TE_OK;
}

extern "C" te_status te_set_demands(te_handle* h, const double* D, int32_t in_is_device) {
    if (!h || !D) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const int K = h->L.K;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    if (!in_is_device) {
        for (int c = 0; c < K; ++c)
            if (!(D[c] > 0.0) || !isfinite(D[c])) return h->fail(TE_EINVAL, fmt("demand %lld is not finite and positive", c));
        A(cudaMemcpyAsync(h->dstage, D, sizeof(double) * K, cudaMemcpyHostToDevice, s));
    } else {
        A(cudaMemcpyAsync(h->dstage, D, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
        A(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
        k_check_demands<<<(K + 255) / 256, 256, 0, s>>>(K, h->dstage, h->flag);
        h->launches += 1;
        int bad = 0;
        A(cudaGetLastError());
        A(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        A(cudaStreamSynchronize(s));
        if (ce != cudaSuccess) return h->cuda(ce, "te_set_demands");
        if (bad) return h->fail(TE_EINVAL, "a demand is not finite and positive");
    }
    const long long nd = (long long)h->L.nblocks * h->L.dpb;
    k_set_demands<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(nd, h->L.demand_of, h->dstage, 1.0 / h->scale,
                                                               h->Dn, h->Dc);
    h->launches += 1;
    A(cudaGetLastError());
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_set_demands");
}

extern "C" te_status te_set_capacities(te_handle* h, const double* C, int32_t in_is_device) {
    if (!h || !C) return TE_EINVAL;
    cudaStream_t s = h->stream;
    const int E = h->L.E;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    if (!in_is_device) {
        for (int e = 0; e < E; ++e)
            if (!(C[e] >= 0.0) || !isfinite(C[e])) return h->fail(TE_EINVAL, fmt("capacity %lld is not finite and >= 0", e));
        A(cudaMemcpyAsync(h->cstage, C, sizeof(double) * E, cudaMemcpyHostToDevice, s));
    } else {
        A(cudaMemcpyAsync(h->cstage, C, sizeof(double) * E, cudaMemcpyDeviceToDevice, s));
        A(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
        k_check_capacities<<<(E + 255) / 256, 256, 0, s>>>(E, h->cstage, h->flag);
        h->launches += 1;
        int bad = 0;
        A(cudaGetLastError());
        A(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        A(cudaStreamSynchronize(s));
        if (ce != cudaSuccess) return h->cuda(ce, "te_set_capacities");
        if (bad) return h->fail(TE_EINVAL, "a capacity is not finite and >= 0");
    }
    k_set_capacities<<<(E + 255) / 256, 256, 0, s>>>(E, h->cstage, 1.0 / h->scale, h->cap_n);
    h->launches += 1;
    A(cudaGetLastError());
    A(cudaStreamSynchronize(s));
    return h->cuda(ce, "te_set_capacities");
}

extern "C" te_status te_gradient(te_handle* h, int64_t iters, int32_t checkpoint_every, double* J_out, double* dJ_dC,
                                 double* dJ_dD, int32_t out_is_device) {
    if (!h || iters < 0 || checkpoint_every < 1 || !dJ_dC || !dJ_dD) return TE_EINVAL;
    if (h->o.adapt_beta || h->o.continuation || !(h->o.gamma < 0.0) || !isfinite(h->o.alpha_target) ||
        h->o.alpha_start != h->o.alpha_target)
        return h->fail(TE_EINVAL, "te_gradient needs the fixed schedule: adapt_beta = 0, continuation = 0, "
                                  "gamma < 0, alpha_start = alpha_target (finite)");
    te_status st = te_reset(h);
    if (st != TE_OK) return st;
    cudaStream_t s = h->stream;
    const te::Layout& L = h->L;
    const size_t ns = (size_t)L.nslots * kLanes, E = (size_t)L.E, ND = (size_t)L.nblocks * L.dpb;
    const size_t state = ns + 2 * E + ND;  // floats: x, u, w, multipliers
    const long long K = iters, ck = checkpoint_every;
    const long long nck = K / ck + 1;
    std::vector<void*> tmp;
    cudaError_t ce = cudaSuccess;
    auto A = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (ce == cudaSuccess) ce = cudaMalloc(&p, bytes > 0 ? bytes : 16);
        if (p) tmp.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void* p : tmp) cudaFree(p);
        tmp.clear();
    };
    float* ckb = (float*)dalloc(sizeof(float) * state * (size_t)nck);
    float* seg = (float*)dalloc(sizeof(float) * state * (size_t)(ck + 1));
    te::AdjointBuffers B{};
    B.xb = (double*)dalloc(sizeof(double) * ns);
    B.ub = (double*)dalloc(sizeof(double) * E);
    B.db = (double*)dalloc(sizeof(double) * E);
    B.Lb = (double*)dalloc(sizeof(double) * E);
    B.Cb = (double*)dalloc(sizeof(double) * E);
    B.qb = (double*)dalloc(sizeof(double) * ns);
    B.wfix = (unsigned long long*)dalloc(sizeof(unsigned long long) * E);
    B.qmax = (unsigned long long*)dalloc(sizeof(unsigned long long));
    B.Db = (double*)dalloc(sizeof(double) * ND);
    B.Uc = (double*)dalloc(sizeof(double) * ND);
    B.acc = (double*)dalloc(sizeof(double));
    {
        // the fixed-point range of the weight adjoint sums: at most (largest
        // number of path-edge incidences on one edge) terms per edge
        std::vector<float> ne((size_t)E);
        A(cudaMemcpy(ne.data(), L.ne_f, sizeof(float) * E, cudaMemcpyDeviceToHost));
        double mx = 1.0;
        for (float v : ne) mx = std::max(mx, (double)v);
        B.deg_bits = 1;
        while (B.deg_bits < 60 && std::ldexp(1.0, B.deg_bits) <= mx) ++B.deg_bits;
    }
    double* gC = out_is_device ? dJ_dC : (double*)dalloc(sizeof(double) * E);
    double* gD = out_is_device ? dJ_dD : (double*)dalloc(sizeof(double) * (size_t)L.K);
    if (ce != cudaSuccess) {
        release();
        cudaGetLastError();
        return h->fail(TE_ENOMEM, "te_gradient: device allocation failed");
    }
    std::vector<te::Scalars> ck_sc((size_t)nck);
    // the handle's state (current rates, prices, weights, multipliers) to and from a slot
    auto save = [&](float* dst) {
        A(cudaMemcpyAsync(dst, h->x + (size_t)h->hsc.xbuf * ns, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(dst + ns, h->u, sizeof(float) * E, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(dst + ns + E, h->w, sizeof(float) * E, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(dst + ns + 2 * E, h->lam, sizeof(float) * ND, cudaMemcpyDeviceToDevice, s));
    };
    auto restore = [&](const float* src, const te::Scalars& sc) {
        h->hsc = sc;
        A(cudaMemcpyAsync(h->x + (size_t)sc.xbuf * ns, src, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(h->u, src + ns, sizeof(float) * E, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(h->w, src + ns + E, sizeof(float) * E, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(h->lam, src + ns + 2 * E, sizeof(float) * ND, cudaMemcpyDeviceToDevice, s));
        A(cudaMemcpyAsync(h->sc, &h->hsc, sizeof(te::Scalars), cudaMemcpyHostToDevice, s));
    };
    // forward, keeping every ck-th state
    for (long long k = 0; k < K && ce == cudaSuccess; ++k) {
        if (k % ck == 0) {
            save(ckb + state * (size_t)(k / ck));
            ck_sc[(size_t)(k / ck)] = h->hsc;
        }
        if ((st = te_solve(h, 1, -1.0, nullptr)) != TE_OK) { release(); return st; }
    }
    const float beta = (float)h->hsc.beta, alpha = (float)h->hsc.alpha;
    A(cudaMemsetAsync(B.ub, 0, sizeof(double) * E, s));
    A(cudaMemsetAsync(B.db, 0, sizeof(double) * E, s));
    A(cudaMemsetAsync(B.Cb, 0, sizeof(double) * E, s));
    A(cudaMemsetAsync(B.wfix, 0, sizeof(unsigned long long) * E, s));
    A(cudaMemsetAsync(B.qb, 0, sizeof(double) * ns, s));
    A(cudaMemsetAsync(B.Db, 0, sizeof(double) * ND, s));
    A(cudaMemsetAsync(B.Uc, 0, sizeof(double) * ND, s));
    A(cudaMemsetAsync(B.acc, 0, sizeof(double), s));
    A(te::adjoint_objective(L, h->x + (size_t)h->hsc.xbuf * ns, h->hsc.alpha, h->scale, B, s));
    h->launches += te::kAdjointObjectiveLaunches;
    // reverse, one checkpoint segment at a time (each recomputed forward first)
    for (long long k0 = K > 0 ? ((K - 1) / ck) * ck : -1; k0 >= 0 && ce == cudaSuccess; k0 -= ck) {
        const long long k1 = std::min(k0 + ck, K);
        restore(ckb + state * (size_t)(k0 / ck), ck_sc[(size_t)(k0 / ck)]);
        for (long long k = k0; k <= k1; ++k) {
            save(seg + state * (size_t)(k - k0));
            if (k < k1 && (st = te_solve(h, 1, -1.0, nullptr)) != TE_OK) { release(); return st; }
        }
        for (long long k = k1 - 1; k >= k0; --k) {
            const float* sk = seg + state * (size_t)(k - k0);
            const float* s1 = seg + state * (size_t)(k + 1 - k0);
            A(te::adjoint_step(L, sk, s1, s1 + ns, sk + ns + E, s1 + ns + 2 * E, beta, alpha, B, s));
            h->launches += te::kAdjointStepLaunches;
        }
    }
    A(te::adjoint_finish(L, h->scale, B, gC, gD, s));
    h->launches += 2;
    double J = 0.0;
    A(cudaMemcpyAsync(&J, B.acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!out_is_device) {
        A(cudaMemcpyAsync(dJ_dC, gC, sizeof(double) * E, cudaMemcpyDeviceToHost, s));
        A(cudaMemcpyAsync(dJ_dD, gD, sizeof(double) * (size_t)L.K, cudaMemcpyDeviceToHost, s));
    }
    A(cudaStreamSynchronize(s));
    release();
    if (ce != cudaSuccess) return h->cuda(ce, "te_gradient");
    if (J_out) *J_out = J;
    return TE_OK;
}

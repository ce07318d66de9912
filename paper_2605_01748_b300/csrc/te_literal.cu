// The update equations of Section 3.3 as printed, run as a multi-block
// iteration on the device: an ablation beside the two-block iteration of the
// library, not a solver (as printed, the capacity and its dual are common to
// every path of an edge and cancel in the rate suggestion, so nothing in the
// iteration sees C_e).  FP64 throughout; one thread per demand, path,
// incidence or edge; the per-edge sums walk a CSC list of each edge's
// incidences in increasing order, so a run is deterministic.
//
// Per iteration, from the rates x, suggestions y and duals of the previous
// one (normalised units, duals per incidence for the consensus terms):
//   dual_dem_c  <- [dual_dem_c + (S_c - D_c)]_+              (dual-updates-dem)
//   dual_cap_e  <- [dual_cap_e + (sum_r y_{e,r} - C_e)]_+     (dual-updates-cap)
//   dual_con_i  <- [dual_con_i + (x_r - y_i)]_+               (dual-updates-con)
//   dual_neg_r  <- [dual_neg_r - x_r]_+                       (dual-updates-neg)
//   cost_i       = beta (-C_e - x_r) - dual_cap_e' - dual_con_i'  (penalty-b)
//   y_i         <- [(mean_{i in e} cost - cost_i) / beta]_+   (rate-suggestion)
//   x_r         <- w_r (Q_r + U'(S) / beta - (S - D_c + dual_dem_c) + dual_neg_r),
//                  w_r = 1 / (1 + n_r), Q_r = sum_{i in r} (y_i - dual_con_i),
//                  with the previous y and duals; S solves the sum of that
//                  formula over the demand's paths            (rate-computation)
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "te_literal.h"

namespace te {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < 1 ? 1 : b);
}

struct LitDev {
    int K, E;
    long long P, nnz;
    const long long* dpo;   // [K+1]
    const long long* peo;   // [P+1]
    const int* pe;          // [nnz] edge of each incidence
    const int* ipath;       // [nnz] path of each incidence
    const long long* eoff;  // [E+1] CSC offsets
    const int* einc;        // [nnz] incidences of each edge, increasing
    const double* D;        // [K]
    const double* C;        // [E]
    const double* ne;       // [E] incidences per edge
    double alpha, beta;
};

// S_c and the demand dual
__global__ void k_lit_demand_dual(LitDev d, const double* x, const double* dem, double* dem_n) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= d.K) return;
    double S = 0.0;
    for (long long r = d.dpo[c]; r < d.dpo[c + 1]; ++r) S += x[r];
    dem_n[c] = fmax(dem[c] + (S - d.D[c]), 0.0);
}

// per path: non-negativity dual, Q_r from the previous y and consensus
// duals, and the new consensus duals of its incidences
__global__ void k_lit_path(LitDev d, const double* x, const double* y, const double* con, const double* neg,
                           double* con_n, double* neg_n, double* Q) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= d.P) return;
    const double xr = x[r];
    neg_n[r] = fmax(neg[r] - xr, 0.0);
    double q = 0.0;
    for (long long i = d.peo[r]; i < d.peo[r + 1]; ++i) {
        q += y[i] - con[i];
        con_n[i] = fmax(con[i] + (xr - y[i]), 0.0);
    }
    Q[r] = q;
}

// per edge: capacity dual and the mean cost of its incidences
__global__ void k_lit_edge(LitDev d, const double* x, const double* y, const double* con_n, const double* cap,
                           double* cap_n, double* mean) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= d.E) return;
    double Ly = 0.0;
    for (long long k = d.eoff[e]; k < d.eoff[e + 1]; ++k) Ly += y[d.einc[k]];
    const double cn = fmax(cap[e] + (Ly - d.C[e]), 0.0);
    cap_n[e] = cn;
    double sc = 0.0;
    for (long long k = d.eoff[e]; k < d.eoff[e + 1]; ++k) {
        const int i = d.einc[k];
        sc += d.beta * (-d.C[e] - x[d.ipath[i]]) - cn - con_n[i];
    }
    mean[e] = sc / fmax(d.ne[e], 1.0);
}

// per incidence: the rate suggestion
__global__ void k_lit_suggest(LitDev d, const double* x, const double* con_n, const double* cap_n,
                              const double* mean, double* y_n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.nnz) return;
    const int e = d.pe[i];
    const double cost = d.beta * (-d.C[e] - x[d.ipath[i]]) - cap_n[e] - con_n[i];
    y_n[i] = fmax((mean[e] - cost) / d.beta, 0.0);
}

// per demand: the total S of the rate formula and the new rates (from the
// previous duals): S (1 + W) = a + W (D - dual_dem) + W U'(S) / beta with
// W = sum_r w_r, a = sum_r w_r (Q_r + dual_neg_r); closed form at alpha = 0,
// bisection (the right side falls as S grows) otherwise
__global__ void k_lit_rates(LitDev d, const double* Q, const double* neg, const double* dem, double* x) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= d.K) return;
    const long long r0 = d.dpo[c], r1 = d.dpo[c + 1];
    double a = 0.0, W = 0.0;
    for (long long r = r0; r < r1; ++r) {
        const double w = 1.0 / (1.0 + (double)(d.peo[r + 1] - d.peo[r]));
        a += w * (Q[r] + neg[r]);
        W += w;
    }
    const double rhs0 = a + W * (d.D[c] - dem[c]);
    double S;
    if (d.alpha == 0.0) {
        S = (rhs0 + W / d.beta) / (1.0 + W);
    } else {
        double lo = 1e-12, hi = fmax(1.0, fabs(rhs0) + W / d.beta) * 10.0 + 1.0;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            const double f = mid * (1.0 + W) - rhs0 - W * pow(mid, -d.alpha) / d.beta;
            if (f < 0.0) lo = mid; else hi = mid;
        }
        S = 0.5 * (lo + hi);
    }
    const double up = d.alpha > 0.0 ? pow(S, -d.alpha) : 1.0;
    for (long long r = r0; r < r1; ++r) {
        const double w = 1.0 / (1.0 + (double)(d.peo[r + 1] - d.peo[r]));
        x[r] = w * (Q[r] + up / d.beta - (S - d.D[c] + dem[c]) + neg[r]);
    }
}

}  // namespace

te_status literal_run(const te_paths* P, int n_edges, const double* demands, const double* capacities, double alpha,
                      double beta, long long iters, double* x_out, cudaStream_t st, std::string& err) {
    const int K = P->n_demands, E = n_edges;
    const long long NP = P->n_paths, nnz = P->nnz;
    // normalised by the geometric mean of the demands
    double lg = 0.0;
    for (int c = 0; c < K; ++c) lg += log(demands[c]);
    const double scale = exp(lg / (double)K);
    std::vector<double> Dn(K), Cn(E), ne(E, 0.0), x0(NP);
    for (int c = 0; c < K; ++c) Dn[c] = demands[c] / scale;
    for (int e = 0; e < E; ++e) Cn[e] = capacities[e] / scale;
    std::vector<int> ipath(nnz);
    for (long long r = 0; r < NP; ++r)
        for (long long i = P->path_edge_off[r]; i < P->path_edge_off[r + 1]; ++i) ipath[i] = (int)r;
    // CSC: each edge's incidences in increasing order
    std::vector<long long> eoff(E + 1, 0);
    for (long long i = 0; i < nnz; ++i) eoff[P->path_edges[i] + 1]++;
    for (int e = 0; e < E; ++e) eoff[e + 1] += eoff[e];
    std::vector<int> einc(nnz);
    {
        std::vector<long long> at(eoff.begin(), eoff.end() - 1);
        for (long long i = 0; i < nnz; ++i) einc[at[P->path_edges[i]]++] = (int)i;
    }
    for (int e = 0; e < E; ++e) ne[e] = (double)(eoff[e + 1] - eoff[e]);
    // Algorithm 1's start: x = D_c / |P_c|, y = x on every incidence, duals 0
    std::vector<double> y0(nnz);
    for (int c = 0; c < K; ++c) {
        const long long r0 = P->demand_path_off[c], r1 = P->demand_path_off[c + 1];
        for (long long r = r0; r < r1; ++r) x0[r] = Dn[c] / (double)(r1 - r0);
    }
    for (long long i = 0; i < nnz; ++i) y0[i] = x0[ipath[i]];

    std::vector<void*> owned;
    cudaError_t ce = cudaSuccess;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (ce == cudaSuccess) ce = cudaMalloc(&p, bytes > 0 ? bytes : 16);
        if (ce == cudaSuccess) owned.push_back(p);
        return p;
    };
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    auto zero = [&](void* dst, size_t bytes) {
        if (ce == cudaSuccess) ce = cudaMemsetAsync(dst, 0, bytes, st);
    };
    LitDev d{};
    d.K = K;
    d.E = E;
    d.P = NP;
    d.nnz = nnz;
    d.alpha = alpha;
    d.beta = beta;
    long long* dpo = (long long*)alloc(sizeof(long long) * (K + 1));
    long long* peo = (long long*)alloc(sizeof(long long) * (NP + 1));
    int* pe = (int*)alloc(sizeof(int) * nnz);
    int* ip = (int*)alloc(sizeof(int) * nnz);
    long long* eo = (long long*)alloc(sizeof(long long) * (E + 1));
    int* ei = (int*)alloc(sizeof(int) * nnz);
    double* Dd = (double*)alloc(sizeof(double) * K);
    double* Cd = (double*)alloc(sizeof(double) * E);
    double* ned = (double*)alloc(sizeof(double) * E);
    double* x = (double*)alloc(sizeof(double) * NP);
    double* Q = (double*)alloc(sizeof(double) * NP);
    double* neg[2] = {(double*)alloc(sizeof(double) * NP), (double*)alloc(sizeof(double) * NP)};
    double* y[2] = {(double*)alloc(sizeof(double) * nnz), (double*)alloc(sizeof(double) * nnz)};
    double* con[2] = {(double*)alloc(sizeof(double) * nnz), (double*)alloc(sizeof(double) * nnz)};
    double* dem[2] = {(double*)alloc(sizeof(double) * K), (double*)alloc(sizeof(double) * K)};
    double* cap[2] = {(double*)alloc(sizeof(double) * E), (double*)alloc(sizeof(double) * E)};
    double* mean = (double*)alloc(sizeof(double) * E);
    put(dpo, P->demand_path_off, sizeof(long long) * (K + 1));
    put(peo, P->path_edge_off, sizeof(long long) * (NP + 1));
    put(pe, P->path_edges, sizeof(int) * nnz);
    put(ip, ipath.data(), sizeof(int) * nnz);
    put(eo, eoff.data(), sizeof(long long) * (E + 1));
    put(ei, einc.data(), sizeof(int) * nnz);
    put(Dd, Dn.data(), sizeof(double) * K);
    put(Cd, Cn.data(), sizeof(double) * E);
    put(ned, ne.data(), sizeof(double) * E);
    put(x, x0.data(), sizeof(double) * NP);
    put(y[0], y0.data(), sizeof(double) * nnz);
    zero(neg[0], sizeof(double) * NP);
    zero(con[0], sizeof(double) * nnz);
    zero(dem[0], sizeof(double) * K);
    zero(cap[0], sizeof(double) * E);
    if (ce == cudaSuccess) {
        d.dpo = dpo;
        d.peo = peo;
        d.pe = pe;
        d.ipath = ip;
        d.eoff = eo;
        d.einc = ei;
        d.D = Dd;
        d.C = Cd;
        d.ne = ned;
        int cur = 0;
        for (long long it = 0; it < iters && ce == cudaSuccess; ++it) {
            const int nx = cur ^ 1;
            k_lit_demand_dual<<<grid_for(K), kThreads, 0, st>>>(d, x, dem[cur], dem[nx]);
            k_lit_path<<<grid_for(NP), kThreads, 0, st>>>(d, x, y[cur], con[cur], neg[cur], con[nx], neg[nx], Q);
            k_lit_edge<<<grid_for(E), kThreads, 0, st>>>(d, x, y[cur], con[nx], cap[cur], cap[nx], mean);
            k_lit_suggest<<<grid_for(nnz), kThreads, 0, st>>>(d, x, con[nx], cap[nx], mean, y[nx]);
            // the rates from the previous duals (dem[cur], neg[cur]) and Q
            k_lit_rates<<<grid_for(K), kThreads, 0, st>>>(d, Q, neg[cur], dem[cur], x);
            ce = cudaPeekAtLastError();
            cur = nx;
        }
    }
    std::vector<double> xh(NP);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(xh.data(), x, sizeof(double) * NP, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    for (void* p : owned) cudaFree(p);
    if (ce != cudaSuccess) {
        err = std::string("te_literal_run: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return ce == cudaErrorMemoryAllocation ? TE_ENOMEM : TE_ECUDA;
    }
    for (long long r = 0; r < NP; ++r) x_out[r] = xh[r] * scale;
    return TE_OK;
}

}  // namespace te

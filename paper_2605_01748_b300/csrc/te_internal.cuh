// Internal declarations shared by the libte translation units (not installed).
//
// Device layout ("sliced" incidence).  Demands are sorted by their vector of
// path lengths and grouped into blocks of 32/G demands; demand t of a block
// owns the G adjacent warp lanes t*G .. t*G+G-1 (G = 1, 2 or 4 lanes per
// demand, so that no lane holds more than 8 paths), and path p of the
// demand sits on lane t*G + p%G in slot p/G.  Block b owns flat slots
// slotbase[b] .. slotbase[b+1]-1.  Per flat slot s:
//   x[s*32 + lane]                      rate of that path (FP32, normalised)
//   ids[(row)*32 + lane], row in [rowoff[s], rowoff[s+1])
//                                       edge ids of that path, hop by hop; a
//                                       shorter path (or a missing one) is
//                                       padded with the sentinel id E
// so every warp-wide load of a slot's rate or of one hop of its paths is one
// contiguous 128 B (rates) or 64 B (16-bit ids) transaction.  Per-demand
// values (demand, path count, multiplier) are stored once per lane, i.e.
// repeated on the G lanes of a demand.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace te {

constexpr int kLanes = 32;
constexpr int kMaxPaths = 32;     // paths per demand
constexpr int kMaxHops = 255;     // edges per path
constexpr int kMaxPathsPerLane = 8;
#ifndef TE_ITER_THREADS
#define TE_ITER_THREADS 1024
#endif
constexpr int kIterThreads = TE_ITER_THREADS;
constexpr int kIterWarps = kIterThreads / 32;
constexpr int kTraceWidth = 5;

// Solver scalars, kept in device memory between launches.
struct Scalars {
    double beta;
    double alpha;
    double r, s;
    long long iter_total;
    long long iter_alpha;
    int converged;     // stop rule fired during the last launch
    int stop_reason;   // 4, 8, 16 (see te.h)
    long long iters_run;  // iterations run by the last launch
    int xbuf;          // which of the two rate buffers holds the iterate
    int pad;
};

struct Options {
    double alpha_target, alpha_start, alpha_step, alpha_max;
    double gamma, A, C;
    int adapt_beta, continuation;
    int withhold_cta;  // test hook: this CTA never arrives at the barrier (-1: none)
};

struct Layout {
    int E;               // edges
    int K;               // demands
    long long P, nnz;    // user paths and incidences
    int nblocks;         // ceil(K / 32)
    long long nslots;    // flat slots
    long long nrows;     // padded id rows (32 ids each)
    int id_bytes;        // 2 (uint16) or 4 (int32)
    int kmax;            // largest paths-per-demand
    int G;               // lanes per demand (1, 2, 4)
    int kl;              // largest paths per lane (<= 8)
    // device arrays
    const void* ids;             // [nrows*32]
    const unsigned* rowoff;      // [nslots+1]
    const int* slotbase;         // [nblocks+1]
    const float* Dn;             // [nblocks*32] normalised demand of the lane's demand, 0 on padding
    const unsigned char* np;     // [nblocks*32] paths of the lane's demand
    const int* lane_demand;      // [nblocks*32] user demand index, -1 on padding
    const long long* slot_path;  // [nslots*32] user path index, -1 on padding
    const float* cap_n;          // [E] normalised capacity
    const float* ne_f;           // [E] paths through the edge
    const float* inv_ne;         // [E] 1/ne (0 if unused)
};

// Arguments of the persistent iteration kernel.
struct IterArgs {
    Layout L;
    Options o;
    float* x;              // [nslots*32] in/out
    float* u;              // [E] scaled prices, in/out
    float* w;              // [E] u + d (gather weights), in/out
    float* loads;          // [3*E] edge-load accumulators (triple buffered)
    double* part;          // [2*grid*4] per-CTA residual partials
    unsigned* barrier;     // grid barrier counter (zeroed before launch)
    int* status;           // device status word (0 ok)
    Scalars* sc;           // in/out
    double* trace;         // [trace_cap*5] ring
    long long trace_cap;
    const int* cta_blk;    // [grid+1] block range of each CTA
    float* lam;            // [nblocks*32] previous multiplier lambda = beta*nu of each demand
    unsigned* ctr;         // [4] scratch counters (zeroed before launch)
    long long max_iters;
    long long timeout_ns;  // bound on every grid-wide wait
};

// Device status codes (mirror te_status).
constexpr int kStatusTimeout = 4;
constexpr int kStatusNumeric = 5;

// Launchers (host side), defined in te_iter.cu / te_proj.cu / te_gap.cu.
size_t iter_smem_bytes(int E);
cudaError_t iter_occupancy(int id_bytes, int kl, int G, int E, int* blocks_per_sm);
cudaError_t launch_iter(const IterArgs& a, int grid, cudaStream_t st);
cudaError_t launch_init_x(const Layout& L, float* x, cudaStream_t st);

// Feasibility projection (Algorithm 2) of a copy x (sliced layout, in place).
// The projection's sums (demand totals, edge loads, remainders, histograms)
// are FP64 so that the violation tests see the loads of the FP32 rates
// without accumulation error.
struct ProjScratch {
    double* S;           // [nblocks*32] demand totals (repeated on the demand's lanes)
    double* loads;       // [E]
    unsigned char* viol; // [E] 1 if L_e > C_e
    int* vidx;           // [E] compact index of violated edges or -1
    int* nviol;          // [1]
    double* hist;        // [E*256] radix-select histograms
    unsigned long long* prefix;  // [E] selected key prefix per violated edge
    double* rem;         // [E] remaining violation per violated edge
    unsigned char* Cp;   // [nslots*32] violated edges per path
};
cudaError_t launch_project(const Layout& L, float* x, float alpha, const ProjScratch& s, cudaStream_t st);
constexpr int kProjectLaunches = 26;  // kernels launch_project issues

// Gather a sliced array to caller path order, times scale.
cudaError_t launch_to_user(const Layout& L, const float* x, float* out, float scale, cudaStream_t st);
cudaError_t launch_from_user(const Layout& L, const float* in, float* x, float inv_scale, cudaStream_t st);

// Duality gap terms of a feasible sliced x (normalised) at prices
// p = beta*u: acc[0] += sum_c U(S_c), acc[1] += sum_c max_S [U(S) - pi_c S],
// acc[2] += sum_e p_e C_e, all in caller units (acc zeroed by the caller).
// Dc: caller-unit demand of each lane (0 on padding lanes).
cudaError_t launch_gap_impl(const Layout& L, const float* x, const float* u, double beta, double alpha,
                            double scale, const double* Dc, double* acc, cudaStream_t st);

// p_out[e] = pscale * u[e] (FP64).
cudaError_t launch_prices(int E, const float* u, double pscale, double* p_out, cudaStream_t st);

}  // namespace te

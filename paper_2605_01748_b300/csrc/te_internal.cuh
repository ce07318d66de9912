// Internal declarations shared by the libte translation units (not installed).
//
// Device layout ("sliced" incidence).  Demands are sorted by their vector of
// path lengths and grouped into blocks of 32/G demands; demand t of a block
// owns the G adjacent warp lanes t*G .. t*G+G-1 (G = 1, 2, 4 or 8 lanes per
// demand, so that no lane holds more than 4 paths), and path p of the
// demand sits on lane t*G + p%G in slot p/G.  Block b owns flat slots
// slotbase[b] .. slotbase[b+1]-1.  Per flat slot s:
//   x[s*32 + lane]                      rate of that path (FP32, normalised)
//   ids[(row)*32 + lane], row in [rowoff[s], rowoff[s+1])
//                                       edge ids of that path, hop by hop; a
//                                       shorter path (or a missing one) is
//                                       padded with the sentinel id E
// so every warp-wide load of a slot's rates or of one hop of its paths is one
// contiguous 128 B (rates) or 64 B (16-bit ids) transaction, and the rows of
// a whole block are one contiguous range that the warp copies into shared
// memory with 16-byte asynchronous copies.  Per-demand values (demand, path count, multiplier) are
// indexed by demand slot d = b*dpb + t.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace te {

constexpr int kLanes = 32;
constexpr int kMaxPaths = 32;     // paths per demand
constexpr int kMaxHops = 255;     // edges per path
constexpr int kMaxPathsPerLane = 4;
// The iteration kernel runs 20 warps per SM: 96 registers per thread fit
// the register file, and two staging buffers of 40 rows per warp, the load
// histograms and the gather weights fit the 227 KB of shared memory for up
// to about 10,000 edges (blocks longer than 40 rows, 0.03 % on the
// 1500-node workload, read their ids from global memory).  The batch
// kernel stages up to 48 rows.
#ifndef TE_ITER_THREADS
#define TE_ITER_THREADS 640
#endif
constexpr int kIterThreads = TE_ITER_THREADS;
constexpr int kIterWarps = kIterThreads / 32;
#ifndef TE_ITER_STAGE_ROWS
#define TE_ITER_STAGE_ROWS 40
#endif
constexpr int kIterStageRows = TE_ITER_STAGE_ROWS;  // rows of 16-bit ids per staging buffer of the iteration kernel
constexpr int kStageRows = 48;      // the same for the batch kernel (3 KB)
constexpr int kTraceWidth = 5;
constexpr int kPartWidth = 8;  // doubles per CTA in IterArgs::part (5 used)

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
    double balance_floor;  // balancing only while max(r, s) exceeds it
    double gamma_max;      // > 0: convergence also needs max_e n_e |d_e| / C_e <= gamma_max
    double beta_cap;       // upper bound of beta (beta_max * beta0, or 1e30)
    int adapt_beta, continuation;
    int deterministic;  // 1: exact fixed-point load histograms; 0: FP32 shared atomics
    int withhold_cta;  // test hook: this CTA never arrives at the barrier (-1: none)
};

// Per-block metadata record: first slot, first id row, rows of slots 0..3
// (8 bits each), number of slots.
struct BlockMeta {
    unsigned s0, row0, counts, kb;
};

struct Layout {
    int E;               // edges
    int K;               // demands
    long long P, nnz;    // user paths and incidences
    int nblocks;         // blocks of dpb demands
    int dpb;             // demands per block (32 / G)
    long long nslots;    // flat slots
    long long nrows;     // padded id rows (32 ids each)
    int id_bytes;        // 2 (uint16) or 4 (int32)
    int kmax;            // largest paths-per-demand
    int G;               // lanes per demand (1, 2, 4, 8)
    int kl;              // largest paths per lane (<= 4)
    int max_block_rows;  // largest rows of one block
    // device arrays
    const void* ids;             // [nrows*32]
    const unsigned* rowoff;      // [nslots+1]
    const int* slotbase;         // [nblocks+1]
    const BlockMeta* blkmeta;    // [nblocks]
    const unsigned* hops;        // [nblocks*32] hop counts of lane l's paths, slot j in bits 8j..8j+7
    const float* Dn;             // [nblocks*dpb] normalised demand, 0 on padding
    const unsigned char* np;     // [nblocks*dpb] paths of the demand
    const int* demand_of;        // [nblocks*dpb] caller demand index, -1 on padding
    const long long* slot_path;  // [nslots*32] caller path index, -1 on padding
    const float* cap_n;          // [E] normalised capacity
    const float* ne_f;           // [E] paths through the edge
    const float* inv_ne;         // [E] 1/ne (0 if unused)
};

// Arguments of the persistent iteration kernel.
struct IterArgs {
    Layout L;
    Options o;
    float* x;              // [2][nslots*32] rate buffers, in/out
    float* u;              // [E] scaled prices, in/out
    float* w;              // [E] u + d (gather weights), in/out
    float* u_next;         // [E] scratch: prices published for a beta rescale
    float* w_next;         // [E] scratch: gather weights published each iteration
    uint2* loads;          // [grid*E] per-CTA partial edge loads (fixed point: 2^-12 and 2^-24
                           // units; FP32 in the first half of each pair's words when not deterministic)
    double* part;          // [2*grid*kPartWidth] per-CTA residual partials: sums of
                           // (x'-x)^2, x'^2, n x'^2, n_e d_e^2 and the largest n_e |d_e| / C_e
    unsigned* barrier;     // grid barrier counter (zeroed before launch)
    int* status;           // device status word (0 ok)
    Scalars* sc;           // in/out
    double* trace;         // [trace_cap*5] ring
    long long trace_cap;
    float* lam;            // [nblocks*dpb] previous multiplier lambda = beta*nu of each demand
    long long max_iters;
    long long timeout_ns;  // bound on every wait (the grid barriers)
    long long xstride;     // floats between the two rate buffers (0: nslots*32)
    // wide-edge mode (instances whose per-edge arrays do not fit a CTA's
    // shared memory): each CTA's load histogram, one 64-bit fixed-point word
    // per edge in units of 2^-24, and its copy of the gather weights live in
    // global memory; nullptr otherwise
    unsigned long long* hist64;  // [grid*(E+1)]
    float* wpriv;                // [grid*(E+1)]
};

// Device status codes (mirror te_status).
constexpr int kStatusTimeout = 4;
constexpr int kStatusNumeric = 5;

// Launchers (host side), defined in te_iter.cu / te_proj.cu / te_gap.cu.
size_t iter_smem_bytes(int E, int grid, bool det);
// The same for the wide-edge mode (staging buffers for ids of id_bytes
// bytes, and the price slice).
size_t iter_smem_bytes_wide(int E, int grid, int id_bytes);
cudaError_t iter_occupancy(int G, bool det, int E, int grid_hint, int* blocks_per_sm);
cudaError_t iter_occupancy_wide(int G, int id_bytes, int E, int grid_hint, int* blocks_per_sm);
cudaError_t launch_iter(const IterArgs& a, int grid, cudaStream_t st);
// Several independent instances in one cooperative launch of the iteration
// kernel (deterministic loads): instance i runs on CTAs i*group ..
// i*group+group-1 with the arguments args_dev[i] (device array of n).
cudaError_t launch_iter_grouped(const IterArgs* args_dev, int n, int group, int G, int E, cudaStream_t st);
cudaError_t launch_init_x(const Layout& L, float* x, cudaStream_t st);

// Duality gap terms of a feasible sliced x (normalised) at prices
// p = beta*u: acc[0] = sum_c U(S_c), acc[1] = sum_c max_S [U(S) - pi_c S],
// acc[2] = sum_e p_e C_e, all in caller units.
// Dc: caller-unit demand of each demand slot (0 on padding).
// The sums are deterministic: per-CTA partials in slots (gap_slot_count(L)
// pairs of doubles, no initial value needed) added in a fixed order.
size_t gap_slot_count(const Layout& L);
cudaError_t launch_gap_impl(const Layout& L, const float* x, const float* u, double beta, double alpha,
                            double scale, const double* Dc, double* acc, double* slots, cudaStream_t st);
constexpr int kGapLaunches = 3;


// p_out[e] = pscale * u[e] (FP64).
cudaError_t launch_prices(int E, const float* u, double pscale, double* p_out, cudaStream_t st);

}  // namespace te

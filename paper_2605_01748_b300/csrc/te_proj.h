// Feasibility steps (Algorithm 2, Section 3.5, and proportional scaling) and
// the gathers between the sliced layout and the caller's path order: host
// declarations of the kernels in te_proj.cu.  Internal; the iteration kernel
// does not use them.
#pragma once

#include "te_internal.cuh"

namespace te {

// Feasibility projection (Algorithm 2) of a copy x (sliced layout, in place).
// Demand totals and remainders are FP64; the edge loads and radix-select
// histograms are exact 64-bit integer sums of the FP32 rates in units of
// 2^-40 (order-free, so the projection is deterministic).
struct ProjScratch {
    double* S;           // [nblocks*dpb] demand totals
    unsigned long long* loads;  // [E] fixed point, rates rounded up
    unsigned char* viol; // [E] 1 if L_e > C_e
    int* vidx;           // [E] compact index of violated edges or -1
    int* nviol;          // [1]
    unsigned long long* hist;   // [E*256] radix-select histograms, fixed point, rates rounded down
    unsigned long long* prefix;  // [E] selected key prefix per violated edge
    double* rem;         // [E] remaining violation per violated edge
    unsigned char* Cp;   // [nslots*32] violated edges per path
    double* score;       // [nblocks*dpb + 256] alpha log(S_c scale) per demand, then log(0..255)
    unsigned long long* vtotal;  // [3] violated incidences counted; fill cursors of entries and paths
    uint4* vlist;        // [vcap] violated incidences, then plist (one allocation, grown by launch_project
                         // as needed; the owner frees vlist)
    uint4* plist;        // [vcap] paths with violated incidences: first entry, count, sliced position
    unsigned long long vcap;
};
// alpha and scale (the caller-unit scale of x) form the paths' score keys.
// *launched (may be NULL) receives the number of kernels launched:
// kProjectLaunches, one more when the list of violated incidences grew.
cudaError_t launch_project(const Layout& L, float* x, double alpha, double scale, ProjScratch& s,
                           cudaStream_t st, int* launched);
constexpr int kProjectLaunches = 27;

// Proportional feasibility scaling (not in the paper): x <- max(x, 0); every
// demand with S_c > D_c scaled by D_c / S_c; then every path by the smallest
// min(1, C_e / L_e) over its edges.  Uses S, loads and rem of the scratch.
cudaError_t launch_project_scale(const Layout& L, float* x, const ProjScratch& s, cudaStream_t st);
constexpr int kProjectScaleLaunches = 5;

// Gather a sliced array to caller path order, times scale.
cudaError_t launch_to_user(const Layout& L, const float* x, float* out, float scale, cudaStream_t st);
cudaError_t launch_from_user(const Layout& L, const float* in, float* x, float inv_scale, cudaStream_t st);

}  // namespace te

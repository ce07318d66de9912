// Reverse-mode pass of te_gradient (te_adjoint.cu): host declarations.
// Internal; the iteration kernel does not use them.
#pragma once

#include "te_internal.cuh"

namespace te {

// Reverse-mode step of one fixed-schedule iteration (te_adjoint.cu): FP64
// adjoints of the rates (per path lane of the sliced layout), of the edge
// prices u and differences d, of the loads, capacities and demands.  The
// adjoint of the gather weights w is summed per edge as exact 64-bit
// fixed-point integers (wfix) of the paths' terms qb, on a power-of-two
// scale set by the step's largest |qb| (qmax) and by deg_bits, so that the
// sums do not depend on the order of the additions.
struct AdjointBuffers {
    double* xb;    // [nslots*32]
    double* ub;    // [E]
    double* db;    // [E]
    double* Lb;    // [E]
    double* Cb;    // [E]
    double* qb;    // [nslots*32] the step's weight adjoint term of each path (0 off the active set)
    unsigned long long* wfix;  // [E] fixed-point sums of qb per edge, zero between steps
    unsigned long long* qmax;  // [1] bits of the step's largest |qb| (a non-negative double)
    double* Db;    // [nblocks*dpb]
    double* Uc;    // [nblocks*dpb] the objective's term of each demand slot (0 on padding)
    double* acc;   // [1] objective
    int deg_bits;  // bits of the largest number of path-edge incidences on one edge, plus one
};
// xk, wk: rates and gather weights entering the iteration; x1, uk1, lam1:
// rates, prices and per-demand multipliers (beta nu) it produced.
cudaError_t adjoint_step(const Layout& L, const float* xk, const float* x1, const float* uk1, const float* wk,
                         const float* lam1, float beta, float alpha, AdjointBuffers& B, cudaStream_t st);
// J of the rates x into acc (the demands' terms summed in a fixed order) and
// its adjoint into xb
cudaError_t adjoint_objective(const Layout& L, const float* x, double alpha, double scale, AdjointBuffers& B,
                              cudaStream_t st);
// the initial state's dependence on the demands, then the gradients in
// caller order and units (gC [E], gD [K], device)
cudaError_t adjoint_finish(const Layout& L, double scale, AdjointBuffers& B, double* gC, double* gD,
                           cudaStream_t st);
constexpr int kAdjointStepLaunches = 4;
constexpr int kAdjointObjectiveLaunches = 2;

}  // namespace te

// Duality gap of a feasible allocation (FP64), for te_gap.
//
// For edge prices p_e >= 0 the Lagrangian dual of the TE problem (Eqs. 1-4)
//   g(p) = sum_e p_e C_e + sum_c max_{0 <= S <= D_c} [U_alpha(S) - pi_c S],
//   pi_c = min_{r in P_c} sum_{e in r} p_e,
// bounds the optimum from above (weak duality); with Slater's point
// (Appendix C, Part I (b)) the bound is tight at the optimum.  The kernel
// evaluates, in the caller's units, sum_c U_alpha(S_c) of the allocation and
// the demand terms of g at p_e = beta u_e (scaled by scale^-alpha, since U'
// scales as S^-alpha); the edge term is added by a second small kernel.
#include <math.h>
#include <stdint.h>

#include "te_internal.cuh"

namespace te {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double utility(double S, double alpha) {
    if (alpha == 1.0) return log(S);
    return (pow(S, 1.0 - alpha) - 1.0) / (1.0 - alpha);
}

// max over 0 <= S <= D of U_alpha(S) - pi S
__device__ __forceinline__ double conj_term(double D, double pi, double alpha) {
    double S;
    if (alpha == 0.0) S = pi < 1.0 ? D : 0.0;
    else if (pi <= 0.0) S = D;
    else S = fmin(D, exp(-log(pi) / alpha));
    if (S <= 0.0) return utility(0.0, alpha);
    return utility(S, alpha) - pi * S;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename IdT>
__global__ void k_gap_demands(Layout L, const float* x, const float* u, double pscale, double alpha,
                              double scale, const double* Dc, double* acc) {
    const IdT* ids = static_cast<const IdT*>(L.ids);
    const int DPB = L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double pr = 0.0, du = 0.0;
    if (i < (long long)L.nblocks * DPB) {
        const int b = (int)(i / DPB), t = (int)(i % DPB);
        const int np = L.np[i];
        if (np > 0) {
            const int s0 = L.slotbase[b];
            double S = 0.0, pi = INFINITY;
            for (int p = 0; p < np; ++p) {
                const int lane = t * L.G + p % L.G;
                const size_t sl = (size_t)(s0 + p / L.G);
                S += (double)x[sl * kLanes + lane];
                double q = 0.0;
                for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                    const IdT id = ids[(size_t)r * kLanes + lane];
                    if ((int)id != L.E) q += (double)u[id];
                }
                pi = fmin(pi, q);
            }
            pr = utility(S * scale, alpha);
            du = conj_term(Dc[i], pi * pscale, alpha);
        }
    }
    pr = warp_sum(pr);
    du = warp_sum(du);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], pr);
        atomicAdd(&acc[1], du);
    }
}

// sum_e p_e C_e with p_e = pscale * u_e and C_e = scale * cap_n[e]
__global__ void k_gap_edges(Layout L, const float* u, double pscale, double scale, double* acc) {
    double v = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.E; e += gridDim.x * blockDim.x)
        v += pscale * (double)u[e] * scale * (double)L.cap_n[e];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[2], v);
}

}  // namespace

// acc[0] = primal sum_c U(S_c), acc[1] = sum_c conj terms, acc[2] = sum_e p_e C_e
// Dc: caller-unit demands in lane order (double), u: scaled prices.
cudaError_t launch_gap_impl(const Layout& L, const float* x, const float* u, double beta, double alpha,
                            double scale, const double* Dc, double* acc, cudaStream_t st) {
    // p = beta * u in normalised units; in caller units U' scales by scale^-alpha
    const double pscale = beta * pow(scale, -alpha);
    const long long nd = (long long)L.nblocks * L.dpb;
    const unsigned g = (unsigned)((nd + kThreads - 1) / kThreads);
    if (L.id_bytes == 2)
        k_gap_demands<uint16_t><<<g, kThreads, 0, st>>>(L, x, u, pscale, alpha, scale, Dc, acc);
    else
        k_gap_demands<int32_t><<<g, kThreads, 0, st>>>(L, x, u, pscale, alpha, scale, Dc, acc);
    k_gap_edges<<<64, kThreads, 0, st>>>(L, u, pscale, scale, acc);
    return cudaGetLastError();
}

}  // namespace te

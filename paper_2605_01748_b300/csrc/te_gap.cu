// Duality gap of a feasible allocation (FP64, with the sums over a demand's
// paths and their edges in pairs of FP32 numbers of about 48 bits), for
// te_gap.
//
// For edge prices p_e >= 0 the Lagrangian dual of the TE problem (Eqs. 1-4)
//   g(p) = sum_e p_e C_e + sum_c max_{0 <= S <= D_c} [U_alpha(S) - pi_c S],
//   pi_c = min_{r in P_c} sum_{e in r} p_e,
// bounds the optimum from above (weak duality); with Slater's point
// (Appendix C, Part I (b)) the bound is tight at the optimum.  The kernels
// evaluate, in the caller's units, sum_c U_alpha(S_c) of the allocation and
// the demand terms of g at p_e = beta u_e (scaled by scale^-alpha, since U'
// scales as S^-alpha), and the edge term sum_e p_e C_e.
//
// Deterministic: every CTA writes its partial sums to a slot of its own (no
// atomics), and one CTA adds the slots in a fixed order, so two calls on the
// same state return the same bits.
#include <math.h>
#include <stdint.h>

#include "te_internal.cuh"

namespace te {
namespace {

constexpr int kThreads = 256;
constexpr int kEdgeCtas = 64;

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

// (hi, lo) += v as an unevaluated FP32 pair: two-sum of hi and v, the
// rounding error added into lo
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float t = hi + v, bv = t - hi;
    lo += (hi - (t - bv)) + (v - bv);
    hi = t;
}
// hi + lo unchanged, |lo| at most half an ulp of hi (fast two-sum; |hi| >=
// |lo| holds for the sums above)
__device__ __forceinline__ void normalise(float& hi, float& lo) {
    const float t = hi + lo;
    lo = lo - (t - hi);
    hi = t;
}

// CTA-wide sums of (a, b) in a fixed order: lanes by a butterfly, warps in
// warp order on thread 0 (the result is valid on thread 0).
__device__ __forceinline__ void cta_sum2(double& a, double& b) {
    __shared__ double red[2][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
    }
}

// One thread per demand slot: slot[2*cta] = sum of U(S_c), slot[2*cta+1] =
// sum of the conjugate terms.
template <typename IdT>
__global__ void k_gap_demands(Layout L, const float* x, const float* u, double pscale, double alpha,
                              double scale, const double* Dc, double* slots) {
    const IdT* ids = static_cast<const IdT*>(L.ids);
    const int DPB = L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double pr = 0.0, du = 0.0;
    if (i < (long long)L.nblocks * DPB) {
        const int b = (int)(i / DPB), t = (int)(i % DPB);
        const int np = L.np[i];
        if (np > 0) {
            const int s0 = L.slotbase[b];
            // The sums below are unevaluated pairs hi + lo of FP32 numbers
            // (the rates and prices are FP32): each addition is split exactly
            // into its rounded sum and its rounding error (Knuth's two-sum),
            // the errors added into lo; a pair is then normalised (|lo| at
            // most half an ulp of hi), so that pairs compare in the order of
            // their values.  About 48 bits, near FP64, on the FP32 units:
            // FP64 is a small fraction of them on this part, and these sums
            // are most of the kernel's work.
            float Sh = 0.f, Sl = 0.f, pih = INFINITY, pil = 0.f;
            for (int p = 0; p < np; ++p) {
                const int lane = t * L.G + p % L.G;
                const size_t sl = (size_t)(s0 + p / L.G);
                two_sum_add(Sh, Sl, x[sl * kLanes + lane]);
                float hi = 0.f, lo = 0.f;  // the path's price sum
                for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                    const IdT id = ids[(size_t)r * kLanes + lane];
                    if ((int)id != L.E) two_sum_add(hi, lo, u[id]);
                }
                normalise(hi, lo);
                if (hi < pih || (hi == pih && lo < pil)) {
                    pih = hi;
                    pil = lo;
                }
            }
            normalise(Sh, Sl);
            const double S = (double)Sh + (double)Sl, pi = (double)pih + (double)pil;
            pr = utility(S * scale, alpha);
            du = conj_term(Dc[i], pi * pscale, alpha);
        }
    }
    cta_sum2(pr, du);
    if (threadIdx.x == 0) {
        slots[2 * blockIdx.x] = pr;
        slots[2 * blockIdx.x + 1] = du;
    }
}

// sum_e p_e C_e with p_e = pscale * u_e and C_e = scale * cap_n[e]; kEdgeCtas
// CTAs, each writing its partial to slot[2*cta+1] (slot[2*cta] = 0).
__global__ void k_gap_edges(Layout L, const float* u, double pscale, double scale, double* slots) {
    double a = 0.0, v = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.E; e += gridDim.x * blockDim.x)
        v += pscale * (double)u[e] * scale * (double)L.cap_n[e];
    cta_sum2(a, v);
    if (threadIdx.x == 0) {
        slots[2 * blockIdx.x] = 0.0;
        slots[2 * blockIdx.x + 1] = v;
    }
}

// One CTA: acc[0] = sum of the primal slots of the demand CTAs, acc[1] = sum
// of their conjugate slots, acc[2] = sum of the edge slots; each thread adds
// a fixed stride of slots, then the threads' sums are combined in thread
// order.
__global__ void k_gap_finish(int nd, int ne, const double* dslots, const double* eslots, double* acc) {
    __shared__ double red[3][kThreads];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nd; i += kThreads) {
        a += dslots[2 * i];
        b += dslots[2 * i + 1];
    }
    for (int i = threadIdx.x; i < ne; i += kThreads) c += eslots[2 * i + 1];
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    red[2][threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int i = 0; i < kThreads; ++i) {
            sa += red[0][i];
            sb += red[1][i];
            sc += red[2][i];
        }
        acc[0] = sa;
        acc[1] = sb;
        acc[2] = sc;
    }
}

}  // namespace

size_t gap_slot_count(const Layout& L) {
    const long long nd = (long long)L.nblocks * L.dpb;
    return (size_t)((nd + kThreads - 1) / kThreads) + kEdgeCtas;
}

// acc[0] = primal sum_c U(S_c), acc[1] = sum_c conj terms, acc[2] = sum_e p_e C_e
// Dc: caller-unit demands in lane order (double), u: scaled prices; slots:
// gap_slot_count(L) pairs of doubles of scratch.
cudaError_t launch_gap_impl(const Layout& L, const float* x, const float* u, double beta, double alpha,
                            double scale, const double* Dc, double* acc, double* slots, cudaStream_t st) {
    // p = beta * u in normalised units; in caller units U' scales by scale^-alpha
    const double pscale = beta * pow(scale, -alpha);
    const long long nd = (long long)L.nblocks * L.dpb;
    const unsigned g = (unsigned)((nd + kThreads - 1) / kThreads);
    if (L.id_bytes == 2)
        k_gap_demands<uint16_t><<<g, kThreads, 0, st>>>(L, x, u, pscale, alpha, scale, Dc, slots);
    else
        k_gap_demands<int32_t><<<g, kThreads, 0, st>>>(L, x, u, pscale, alpha, scale, Dc, slots);
    double* eslots = slots + 2 * (size_t)g;
    k_gap_edges<<<kEdgeCtas, kThreads, 0, st>>>(L, u, pscale, scale, eslots);
    k_gap_finish<<<1, kThreads, 0, st>>>((int)g, kEdgeCtas, slots, eslots, acc);
    return cudaGetLastError();
}

}  // namespace te

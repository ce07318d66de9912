// Device code shared by the iteration kernels (the single-instance persistent
// kernel and the batch kernel): bounded waits and barriers, reductions, the
// per-demand solve (x-block), asynchronous copies into shared memory, and the
// processing of one block (gather, per-demand split, scatter into the
// CTA's load histogram).  Internal; included by te_iter.cu and te_batch.cu.
#pragma once

#include <math.h>
#include <stdint.h>

#include "te_internal.cuh"

namespace te {
namespace {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch.  Every wait is bounded: after
// timeout_ns the CTA records kStatusTimeout and gives up; a CTA that sees a
// non-zero status also gives up.  Returns false when the barrier failed.
// arrive = false is the test hook of a CTA that withholds its arrival.
__device__ bool grid_sync(unsigned* counter, unsigned target, int* status, long long timeout_ns, bool arrive) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (arrive) atomicAdd(counter, 1u);
        int ok = 1;
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire(counter) < target) {
            if (*(volatile int*)status != 0) { ok = 0; break; }
            if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
                atomicCAS(status, 0, kStatusTimeout);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Residual balancing (Eq. 17): beta times C when r > A s, divided by C when
// s > A r; a step that would leave [kBetaMin, min(kBetaMax, cap)] is not
// taken (1/beta and log beta stay finite FP32 values; cap is the caller's
// bound beta_max * beta0, or kBetaMax).
constexpr double kBetaMin = 1e-30, kBetaMax = 1e30;
__device__ __forceinline__ double balanced_beta(double beta, double r, double s, double A, double C, double cap) {
    double nb = beta;
    if (r > A * s) nb = beta * C;
    else if (s > A * r) nb = beta / C;
    return (nb >= kBetaMin && nb <= fmin(kBetaMax, cap)) ? nb : beta;
}

// Kahan-compensated FP32 accumulation (per-thread partial sums of the
// residual norms; the cross-thread reduction is FP64).  c holds minus the
// low-order part lost so far, so the sum is s - c; for non-negative terms
// the error of the compensated sum is at most about 2 eps times the sum
// (eps = 2^-24), independent of the number of terms.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// A lane's running sums of the residual terms of its warp's blocks (Eqs.
// 15-16): sum (x' - x)^2 compensated (it decides convergence: its terms are
// small differences that shrink by orders of magnitude over a solve), and
// the norms sum x'^2 and sum n_r x'^2 (positive terms of similar size, which
// only scale the residuals) in plain FP32.
struct LaneRes {
    KSum d;
    float x = 0.f, e = 0.f;
};

// Root of A + H nu = (beta nu)^(-1/alpha) in t = log nu on (tlo, thi); the
// demand cap is slack here.  alpha = 1 has the closed-form quadratic root of
// Appendix B.2; other alpha use Newton steps on
// g(t) = log(A + H e^t) + (t + log beta)/alpha, safeguarded by bisection.
// ia = 1/alpha (FP32, computed once per iteration by the caller).
__device__ __forceinline__ float slack_root(float A, float H, float logbeta, float alpha, float ia, float tlo,
                                            float thi, float hint) {
    if (alpha == 1.f) {
        const float ib = __expf(-logbeta);
        const float disc = sqrtf(fmaf(A, A, 4.f * H * ib));
        return A >= 0.f ? 2.f * ib / (A + disc) : (disc - A) / (2.f * H);
    }
    // start from the previous multiplier when it lies inside the bracket
    const float th = hint > 0.f ? __logf(hint) : thi;
    float t = (th > tlo && th < thi) ? th : thi;
    #pragma unroll 1
    for (int it = 0; it < 40; ++it) {
        const float et = __expf(t);
        const float s = fmaf(H, et, A);
        float tn;
        if (s > 0.f) {
            const float ls = __logf(s), lt = (t + logbeta) * ia;
            const float g = ls + lt;
            if (g > 0.f) thi = t; else tlo = t;
            // the step only has to move t towards the root: its quotients
            // may be approximate (the accepted t still solves g(t) = 0)
            const float dg = __fdividef(H * et, s) + ia;
            tn = t - __fdividef(g, dg);
            // g carries the rounding error of its two terms (a few units in
            // the last place of each, and of t + log beta); a Newton step no
            // larger than that error divided by g', or than the tolerance,
            // ends the loop, also where it does not fall strictly inside the
            // bracket (g = 0 exactly, or a step that rounds back to t)
            const float eg = fmaf(1.2e-7f * ia, fabsf(t) + fabsf(logbeta), 4e-7f * fmaxf(1.f, fabsf(ls)));
            if (fabsf(tn - t) <= fmaxf(2e-7f * fmaxf(1.f, fabsf(t)), __fdividef(eg, dg))) { t = tn; break; }
        } else {
            tlo = t;
            tn = 0.5f * (tlo + thi);
        }
        if (!(tn > tlo && tn < thi)) tn = 0.5f * (tlo + thi);
        if (fabsf(tn - t) <= 2e-7f * fmaxf(1.f, fabsf(t))) { t = tn; break; }
        t = tn;
    }
    return __expf(t);
}

// Sums / minimum / all-true over the G adjacent lanes of one demand.  The
// butterfly gives every lane of the group the same value (the additions are
// commutative at each level), so decisions taken on it are group-uniform.
template <int G>
__device__ __forceinline__ float gsum(float v, unsigned gm) {
    if (G >= 2) v += __shfl_xor_sync(gm, v, 1);
    if (G >= 4) v += __shfl_xor_sync(gm, v, 2);
    if (G >= 8) v += __shfl_xor_sync(gm, v, 4);
    return v;
}
template <int G>
__device__ __forceinline__ float gmin(float v, unsigned gm) {
    if (G >= 2) v = fminf(v, __shfl_xor_sync(gm, v, 1));
    if (G >= 4) v = fminf(v, __shfl_xor_sync(gm, v, 2));
    if (G >= 8) v = fminf(v, __shfl_xor_sync(gm, v, 4));
    return v;
}
template <int G>
__device__ __forceinline__ int gall(int v, unsigned gm) {
    if (G >= 2) v &= __shfl_xor_sync(gm, v, 1);
    if (G >= 4) v &= __shfl_xor_sync(gm, v, 2);
    if (G >= 8) v &= __shfl_xor_sync(gm, v, 4);
    return v;
}

// Per-demand x-block in scaled form, the demand's paths spread over G lanes
// (this lane holds KL of them; an[j] == 0 marks an absent slot).  Returns
// nu with x_r = max(0, m_r + nu an_r), where an_r = 1/n_r.
//
// S(nu) = sum_r max(0, m_r + nu an_r) is convex, piecewise linear and
// increasing; the solution is the point where S(nu) meets the target
// T(nu) = min(D, (beta nu)^(-1/alpha)) (alpha > 0; T decreases), or
// min(1/beta, nu_D) with S(nu_D) = D (alpha = 0).  Each step replaces S by
// its supporting line at the current nu (the active paths' sums of m and an)
// and moves to where that line meets T.  The line lies below S, so from any
// start the first step lands at or right of the solution, and from there the
// steps decrease monotonically onto it; the loop ends when the active set at
// the new point equals the one that produced it (then the point is exact).
// nu0 is the previous iteration's multiplier of this demand (a warm start:
// typically the first step is already exact and the second confirms it).
template <int KL, int G>
__device__ __forceinline__ float solve_nu(const float (&m)[KL], const float (&an)[KL], float D,
                                          float inv_beta, float logbeta, float alpha, float inv_alpha, float nu0,
                                          unsigned gm) {
    float nu = nu0;
    if (alpha == 0.f) {
        float S = 0.f;
        #pragma unroll
        for (int j = 0; j < KL; ++j)
            if (an[j] > 0.f) S += fmaxf(0.f, fmaf(inv_beta, an[j], m[j]));
        S = gsum<G>(S, gm);
        if (S <= D) return inv_beta;  // lambda = U'(S) = 1, cap slack
        nu = fminf(nu, inv_beta);
    }
    // the nu at which (beta nu)^(-1/alpha) = D, and its log
    const float tcap = alpha > 0.f ? -alpha * __logf(D) - logbeta : INFINITY;
    const float nucap = alpha > 0.f ? __expf(tcap) : INFINITY;
    unsigned prev = 0u;
    bool descending = false;  // nu is a root computed from a supporting line (an upper bound)
    #pragma unroll 1
    for (int it = 0; it < KL * G + 3; ++it) {
        float A = 0.f, H = 0.f;
        unsigned mask = 0u;
        #pragma unroll
        for (int j = 0; j < KL; ++j) {
            if (an[j] > 0.f && fmaf(nu, an[j], m[j]) > 0.f) {
                A += m[j];
                H += an[j];
                mask |= 1u << j;
            }
        }
        if (descending && gall<G>(mask == prev, gm)) break;  // nu is the root of this line
        A = gsum<G>(A, gm);
        H = gsum<G>(H, gm);
        if (!(H > 0.f)) {
            // nothing active at nu.  While descending this only happens when
            // the root lies on a path's breakpoint and rounding switched the
            // path off: its rate there is zero to rounding, so stop.  At the
            // start, restart from a single-path bound instead (one path
            // alone reaches D there, so S(nu) >= D >= T(nu)).
            if (descending) break;
            float ub = INFINITY;
            #pragma unroll
            for (int j = 0; j < KL; ++j)
                if (an[j] > 0.f) ub = fminf(ub, (D - m[j]) / an[j]);
            nu = gmin<G>(ub, gm);
            continue;
        }
        // where the line meets D.  Beyond nucap (alpha > 0; tested without
        // the quotient, H > 0) the cap is slack and the root is where the
        // line meets (beta nu)^(-1/alpha), below that point
        const float DA = D - A;
        float nn;
        if (DA > nucap * H) nn = slack_root(A, H, logbeta, alpha, inv_alpha, tcap, __logf(DA) - __logf(H), nu);
        else nn = DA / H;
        if (descending && !(nn < nu)) break;  // rounding: no further descent
        nu = nn;
        prev = mask;
        descending = true;
    }
    return nu;
}


// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// one 16-byte asynchronous copy by this thread (both addresses 16-byte
// aligned); copies are grouped per thread and waited for per group
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most the most recent group of this thread is in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// 64-bit integer add into global memory with no value returned (a reduction
// the L2 performs; the caller does not wait for it)
__device__ __forceinline__ void red_add_global_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}
// 32-bit load from a 32-bit shared-memory address
__device__ __forceinline__ uint32_t lds_u32(unsigned addr) {
    unsigned v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
// 16-bit load from a 32-bit shared-memory address
__device__ __forceinline__ uint16_t lds_u16(unsigned addr) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}
// One block (32/G demands, G lanes each, at most 4 paths per lane): gather,
// x-block, scatter.  bids points at the block's first id row, in shared
// memory (STAGED) or in global memory.
// What the per-block code needs besides the block itself: the demand and
// multiplier arrays (indexed by demand slot), the per-block residual terms,
// the per-lane hop counts (HOPS), demands per block and the padding id.
struct BlockCtx {
    const float* Dn;
    float* lam;
    float* blkres;
    const unsigned* hops;
    int dpb;
    uint16_t sentinel;
};

// Per-lane inputs of one block read from global memory: the lane's rates,
// its demand, the demand's multiplier and (HOPS) the hop counts of the
// lane's paths, slot j in bits 8j..8j+7.  Loaded one block ahead of use.
template <int KL = kMaxPathsPerLane>
struct BlockIn {
    float x[KL];
    float D, lam;
    unsigned nb;
};

template <int G, bool HOPS, int KL = kMaxPathsPerLane>
__device__ __forceinline__ BlockIn<KL> load_block_in(const BlockCtx& a, int b, int lane, int s0, int KB,
                                                 const float* __restrict__ xin) {
    BlockIn<KL> in;
    const size_t di = (size_t)b * a.dpb + lane / G;
    in.D = __ldg(&a.Dn[di]);
    in.lam = __ldcg(&a.lam[di]);
    in.nb = HOPS ? __ldg(&a.hops[(size_t)b * kLanes + lane]) : 0u;
    const float* xp = xin + (size_t)s0 * kLanes + lane;
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        in.x[j] = 0.f;
        if (j < KB) in.x[j] = __ldcg(xp + j * kLanes);
    }
    return in;
}

// ACC: the block's residual terms are added into this lane's compensated
// running sums acc (the caller reduces them once per phase, in FP64), else
// summed over the warp and stored per block.  HOPS: the hop counts come with the block's inputs,
// else the gather counts the non-padding ids.  DET: each rate enters the
// load histogram as an exact split fixed-point pair (h_hi, h_lo: two 32-bit
// integer atomics per incidence, order-free); else h_hi is an FP32
// histogram and each rate is added by one FP32 shared atomic per incidence
// (the sum then depends on the order of the atomics in its last bits).
// GH (with DET): the histogram is one 64-bit word per edge in global memory,
// h_hi read as unsigned long long*, and each rate adds the same fixed-point
// value hi * 2^12 + lo (units of 2^-24) by one 64-bit L2 reduction (red:
// no value returned, so the warp does not wait for it); h_lo unused.
// IdT: the layout's edge id type (uint16_t, or uint32_t above 65,534 edges,
// where the hop counts come with the block: HOPS).  KL: the path slots a lane
// can hold (kMaxPathsPerLane; 1 for layouts of one path per lane, where the
// absent slots' loops and registers go away; the arithmetic is the same).
template <int G, bool STAGED, bool ACC, bool HOPS, bool DET, bool GH = false, typename IdT = uint16_t,
          int KL = kMaxPathsPerLane>
__device__ __forceinline__ void process_block(const BlockCtx& a, int b, int lane, const IdT* bids, int s0,
                                              unsigned counts, int KB, const BlockIn<KL>& in,
                                              float* __restrict__ xout, const float* w_s, unsigned* h_hi,
                                              unsigned* h_lo, float inv_beta, float logbeta,
                                              float beta_f, float alpha, float inv_alpha, LaneRes& acc) {
    static_assert(KL >= 1 && KL <= kMaxPathsPerLane, "path slots per lane");
    static_assert(sizeof(IdT) == 2 || (sizeof(IdT) == 4 && HOPS), "32-bit ids come with stored hop counts");
    const IdT sentinel = (IdT)a.sentinel;
    const unsigned gm = G == 1 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const size_t di = (size_t)b * a.dpb + lane / G;
    const float D = in.D;
    const float lam0 = in.lam;
    float xo[KL], m[KL], an[KL];
    #pragma unroll
    for (int j = 0; j < KL; ++j) xo[j] = in.x[j];
    // staged ids: 32-bit shared address of this lane's entry in the block's
    // first row (an explicit shared load per row, no generic addressing)
    const unsigned sb = STAGED ? smem_u32(bids) + (unsigned)sizeof(IdT) * (unsigned)lane : 0u;
    auto id_at = [&](unsigned row) -> IdT {
        if (STAGED) {
            const unsigned at = sb + row * (unsigned)(kLanes * sizeof(IdT));
            if (sizeof(IdT) == 2) return (IdT)lds_u16(at);
            return (IdT)lds_u32(at);
        }
        return __ldg(&bids[(size_t)row * kLanes + lane]);
    };
    unsigned rs = 0;                      // first row of slot j within the block
    unsigned nbits = HOPS ? in.nb : 0u;  // hop count n of slot j's path in bits 8j..8j+7
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        m[j] = 0.f;
        an[j] = 0.f;
        if (j < KB) {
            const unsigned cnt = (counts >> (8 * j)) & 0xffu;
            float q = 0.f;
            int n = HOPS ? (int)((nbits >> (8 * j)) & 0xffu) : 0;
            #pragma unroll 4
            for (unsigned r = 0; r < cnt; ++r) {
                const IdT id = id_at(rs + r);
                q += w_s[id];
                if (!HOPS) n += (id != sentinel);
            }
            if (n > 0) {
                // 1/n by the hardware's approximate reciprocal (within an
                // ulp; measured 3 % less time per iteration than the
                // correctly rounded one)
                an[j] = __fdividef(1.f, (float)n);
                m[j] = fmaf(-q, an[j], xo[j]);
            }
            if (!HOPS) nbits |= (unsigned)n << (8 * j);
            rs += cnt;
        }
    }
    float nu = 0.f;
    if (D > 0.f) {
        nu = solve_nu<KL, G>(m, an, D, inv_beta, logbeta, alpha, inv_alpha, lam0 * inv_beta, gm);
        if ((lane & (G - 1)) == 0) __stcg(&a.lam[di], nu * beta_f);
    }
    // this block's residual terms (at most 4 paths per lane, plain FP32)
    float bd = 0.f, bx = 0.f, be = 0.f;
    float* xq = xout + (size_t)s0 * kLanes + lane;
    rs = 0;
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        if (j < KB) {
            const unsigned cnt = (counts >> (8 * j)) & 0xffu;
            const float xn = an[j] > 0.f ? fmaxf(0.f, fmaf(nu, an[j], m[j])) : 0.f;
            __stcg(xq + j * kLanes, xn);
            const float dx = xn - xo[j];
            bd = fmaf(dx, dx, bd);
            bx = fmaf(xn, xn, bx);
            if (xn != 0.f && !DET) {
                be = fmaf(xn * xn, (float)((nbits >> (8 * j)) & 0xffu), be);
                float* h_f = reinterpret_cast<float*>(h_hi);
                #pragma unroll 8
                for (unsigned r = 0; r < cnt; ++r) atomicAdd(&h_f[id_at(rs + r)], xn);
            } else if (xn != 0.f) {
                // the path's hop count n (n <= 255 hops)
                be = fmaf(xn * xn, (float)((nbits >> (8 * j)) & 0xffu), be);
                // split fixed point: integer part of xn * 2^12 and the
                // remaining fraction in units of 2^-24 (both exact in FP32)
                const float vf = xn * 0x1p12f;
                const float hf = floorf(vf);
                const unsigned hi = (unsigned)hf;
                const unsigned lo = (unsigned)__float2uint_rn((vf - hf) * 0x1p12f);
                // no per-row branch: padding entries (the sentinel id E) add
                // into the unused histogram slot E.  Unrolled by 8 (measured:
                // 1.5-3 % less time per iteration than by 4 or 6)
                if (GH) {
                    unsigned long long* h64 = reinterpret_cast<unsigned long long*>(h_hi);
                    const unsigned long long v = ((unsigned long long)hi << 12) + lo;
                    #pragma unroll 8
                    for (unsigned r = 0; r < cnt; ++r) red_add_global_u64(&h64[id_at(rs + r)], v);
                } else {
                    #pragma unroll 8
                    for (unsigned r = 0; r < cnt; ++r) {
                        const IdT id = id_at(rs + r);
                        atomicAdd(&h_hi[id], hi);
                        atomicAdd(&h_lo[id], lo);
                    }
                }
            }
            rs += cnt;
        }
    }
    if (ACC) {
        // added into the lane's compensated running sums
        acc.d.add(bd);
        acc.x += bx;
        acc.e += be;
    } else {
        // the block's residual terms, summed over the warp in a fixed order
        // and stored per block, so that their totals do not depend on which
        // warp processed which block
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bd += __shfl_xor_sync(0xffffffffu, bd, o);
            bx += __shfl_xor_sync(0xffffffffu, bx, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
        }
        if (lane == 0) {
            float* r = a.blkres + (size_t)b * 3;
            __stcg(&r[0], bd);
            __stcg(&r[1], bx);
            __stcg(&r[2], be);
        }
    }
}

__device__ __forceinline__ unsigned rows_of(unsigned counts) {
    return (counts & 0xffu) + ((counts >> 8) & 0xffu) + ((counts >> 16) & 0xffu) + (counts >> 24);
}

// Per-warp staging buffers of the block pipeline: two adjacent buffers of
// ROWS id rows from base (a block is copied into one while the other is
// processed).  Buffer k is addressed as base + k * ROWS * 32, not through an
// array of two pointers: a pointer array indexed by the alternating buffer
// number would live in local memory and be reloaded for every block.
struct WarpStage {
    uint16_t* base;
};
template <int ROWS, typename IdT = uint16_t>
__device__ __forceinline__ IdT* stage_buf(const WarpStage& ws, int k) {
    return reinterpret_cast<IdT*>(ws.base) + (k ? ROWS * kLanes : 0);
}

// Phase A of one iteration for one warp: takes blocks start + v * stride
// for v = w, w + W, w + 2W, ... < count (w the warp, W the warps of the CTA:
// a fixed interleave, so no counter is shared; the blocks of a CTA are a
// sample of all kinds of blocks, and the warps' totals differ little), brings
// each block's id rows into a staging buffer by asynchronous 16-byte copies
// (every lane a share, one commit group per block) issued one block ahead
// (blocks longer than ROWS read their ids from global memory), loads
// the next block's rates, demands and multipliers into registers while the
// current block is processed, and processes it.  blkmeta, ids and the rate
// buffers are those of the instance.  All copies have landed on return.
//
// Per-lane copies instead of one bulk (TMA) copy per block: the ids of a
// block are one contiguous range of about 1.6 KB, and on the 1500-node
// workload the bulk copy's issue and completion wait cost a warp about 1900
// cycles per block against 6.8 % less time per iteration with cp.async.
//
// ACC (see process_block): the residual terms of the warp's blocks are summed
// per lane into acc (compensated), in the fixed order of the interleave.  HOPS
// and DET: see process_block.  GH, IdT: see process_block (with 32-bit ids a
// warp's two staging buffers take twice the bytes: ws.base must have room).
template <int G, int ROWS, bool ACC, bool HOPS, bool DET, bool GH = false, typename IdT = uint16_t,
          int KL = kMaxPathsPerLane>
__device__ void run_blocks(int start, int stride, int count, const BlockMeta* __restrict__ blkmeta,
                           const IdT* __restrict__ ids, const float* __restrict__ xin,
                           float* __restrict__ xout, const BlockCtx& bc, WarpStage& ws, const float* w_s,
                           unsigned* h_hi, unsigned* h_lo, float inv_beta, float logbeta, float beta_f,
                           float alpha, float inv_alpha, LaneRes& acc) {
    const int lane = threadIdx.x & 31;
    const int none = start + count * stride;  // any index >= none means "no block"
    const int nw = (int)(blockDim.x >> 5);
    int vnext = (int)(threadIdx.x >> 5);
    auto grab = [&]() -> int {
        const int v = vnext;
        vnext += nw;
        return v < count ? start + v * stride : none;
    };
    auto load_meta = [&](int b) -> BlockMeta {
        BlockMeta m{0u, 0u, 0u, 0u};
        if (lane == 0 && b < none) m = blkmeta[b];
        return m;
    };
    // issues the copies of block b into buffer k (the caller commits the
    // group); returns whether the block fits a staging buffer (else it is
    // read from global memory).  The __syncwarp orders every lane's reads
    // of buffer k (the block before last) before the copies overwrite it.
    auto issue = [&](const BlockMeta& m, int k) -> bool {
        const unsigned counts = __shfl_sync(0xffffffffu, m.counts, 0);
        const unsigned row0 = __shfl_sync(0xffffffffu, m.row0, 0);
        const unsigned rows = rows_of(counts);
        if (rows > (unsigned)ROWS || rows == 0) return false;
        __syncwarp();
        const unsigned bytes = rows * kLanes * (unsigned)sizeof(IdT);  // a multiple of 64
        const char* src = reinterpret_cast<const char*>(ids + (size_t)row0 * kLanes);
        const unsigned dst = smem_u32(stage_buf<ROWS, IdT>(ws, k));
        // at most ROWS rows of 64 B: a fixed number of predicated copies per
        // lane (no loop branch)
        constexpr int kCopies = ROWS * kLanes * (int)sizeof(IdT) / (16 * kLanes);
        static_assert(ROWS * (int)sizeof(IdT) % 16 == 0, "a staging buffer is whole 16-byte copies per lane");
        #pragma unroll
        for (int i = 0; i < kCopies; ++i) {
            const unsigned off = 16u * ((unsigned)lane + (unsigned)i * kLanes);
            if (off < bytes) cp_async16(dst + off, src + off);
        }
        return true;
    };
    auto prefetch = [&](int b, const BlockMeta& m) -> BlockIn<KL> {
        const int s0 = (int)__shfl_sync(0xffffffffu, m.s0, 0);
        const int KB = (int)__shfl_sync(0xffffffffu, m.kb, 0);
        BlockIn<KL> in{};
        if (b < none) in = load_block_in<G, HOPS, KL>(bc, b, lane, s0, KB, xin);
        return in;
    };
    int b0 = grab();
    BlockMeta m0 = load_meta(b0);
    int b1 = grab();
    BlockMeta m1 = load_meta(b1);
    int cur = 0;
    bool st0 = b0 < none ? issue(m0, cur) : false;
    cp_async_commit();  // one group per block, empty when nothing was copied
    BlockIn<KL> in0 = prefetch(b0, m0);
    while (b0 < none) {
        const int b2 = grab();
        const BlockMeta m2 = load_meta(b2);
        const bool st1 = b1 < none ? issue(m1, cur ^ 1) : false;
        cp_async_commit();
        const BlockIn<KL> in1 = prefetch(b1, m1);
        const int s0 = (int)__shfl_sync(0xffffffffu, m0.s0, 0);
        const unsigned counts = __shfl_sync(0xffffffffu, m0.counts, 0);
        const int KB = (int)__shfl_sync(0xffffffffu, m0.kb, 0);
        if (st0) {
            // this block's group (all but the newest) has landed for every
            // lane; the __syncwarp makes each lane's copies visible to all
            cp_async_wait_prev();
            __syncwarp();
            process_block<G, true, ACC, HOPS, DET, GH, IdT, KL>(bc, b0, lane, stage_buf<ROWS, IdT>(ws, cur), s0, counts, KB, in0, xout, w_s, h_hi, h_lo,
                                        inv_beta, logbeta, beta_f, alpha, inv_alpha, acc);
        } else {
            const unsigned row0 = __shfl_sync(0xffffffffu, m0.row0, 0);
            process_block<G, false, ACC, HOPS, DET, GH, IdT, KL>(bc, b0, lane, ids + (size_t)row0 * kLanes, s0, counts, KB, in0, xout,
                                         w_s, h_hi, h_lo, inv_beta, logbeta, beta_f, alpha, inv_alpha, acc);
        }
        b0 = b1;
        m0 = m1;
        in0 = in1;
        st0 = st1;
        b1 = b2;
        m1 = m2;
        cur ^= 1;
    }
    cp_async_wait_all();  // (only empty groups can remain)
    __syncwarp();
}

}  // namespace
}  // namespace te

// Persistent iteration kernel of the GATE ADMM loop (Algorithm 1).
//
// One cooperative launch runs many iterations.  Per iteration:
//   phase A (every CTA, one warp per block of 32 demands, one lane per
//            demand): gather the consensus term of each path from the edge
//            weights w_e = u_e + d_e held in shared memory, solve the demand's
//            x-block (Eq. 14 and the sum computation of Appendix B.2), write
//            the new rates, and add each path's new rate into a per-CTA
//            shared-memory histogram of edge loads; then flush the histogram
//            into a global load vector and publish the CTA's FP64 residual
//            partials;
//   one bounded grid-wide barrier;
//   phase B (every CTA, redundantly and identically): the per-edge price
//            update u_e' = max(0, u_e + (L_e - C_e)/n_e) (Eqs. 9/13 after the
//            per-edge collapse of the consensus duals), the residuals r and s
//            (Eqs. 15-16, cross-thread and cross-CTA sums in FP64), residual
//            balancing (Eq. 17), the stop rule (Eq. 18) and
//            alpha-continuation.  Every CTA reads the same loads and partials
//            in the same order, so all of them hold bit-identical prices and
//            take the same decisions without a second barrier.
//
// Rates and prices are FP32.  The per-demand multiplier is kept in scaled
// form nu = lambda / beta, so x_r = max(0, m_r + nu / n_r) with
// m_r = x_r - (1/n_r) sum_{e in r} w_e, and lambda = U'(S) = S^-alpha becomes
// beta nu S^alpha = 1, solved in the log domain (no overflow of S^-alpha at
// large alpha).
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

// Sum of one double over the CTA; every thread receives the result.  The
// reduction order is fixed, so all CTAs obtain identical values from
// identical inputs.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < kIterWarps; ++i) t += red[i];
    return t;
}

// Kahan-compensated FP32 accumulation (per-thread partial sums of the
// residual norms; the cross-thread reduction is FP64).
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Root of A + H nu = (beta nu)^(-1/alpha) in t = log nu on (tlo, thi); the
// demand cap is slack here.  alpha = 1 has the closed-form quadratic root of
// Appendix B.2; other alpha use Newton steps on
// g(t) = log(A + H e^t) + (t + log beta)/alpha, safeguarded by bisection.
__device__ __forceinline__ float slack_root(float A, float H, float logbeta, float alpha, float tlo,
                                            float thi, float hint) {
    if (alpha == 1.f) {
        const float ib = __expf(-logbeta);
        const float disc = sqrtf(fmaf(A, A, 4.f * H * ib));
        return A >= 0.f ? 2.f * ib / (A + disc) : (disc - A) / (2.f * H);
    }
    const float ia = 1.f / alpha;
    // start from the previous multiplier when it lies inside the bracket
    const float th = hint > 0.f ? __logf(hint) : thi;
    float t = (th > tlo && th < thi) ? th : thi;
    #pragma unroll 1
    for (int it = 0; it < 40; ++it) {
        const float et = __expf(t);
        const float s = fmaf(H, et, A);
        float tn;
        if (s > 0.f) {
            const float g = __logf(s) + (t + logbeta) * ia;
            if (g > 0.f) thi = t; else tlo = t;
            const float dg = H * et / s + ia;
            tn = t - g / dg;
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
    return v;
}
template <int G>
__device__ __forceinline__ float gmin(float v, unsigned gm) {
    if (G >= 2) v = fminf(v, __shfl_xor_sync(gm, v, 1));
    if (G >= 4) v = fminf(v, __shfl_xor_sync(gm, v, 2));
    return v;
}
template <int G>
__device__ __forceinline__ int gall(int v, unsigned gm) {
    if (G >= 2) v &= __shfl_xor_sync(gm, v, 1);
    if (G >= 4) v &= __shfl_xor_sync(gm, v, 2);
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
                                          float inv_beta, float logbeta, float alpha, float nu0, unsigned gm) {
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
    // log of the nu at which (beta nu)^(-1/alpha) = D
    const float tcap = alpha > 0.f ? -alpha * __logf(D) - logbeta : INFINITY;
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
        A = gsum<G>(A, gm);
        H = gsum<G>(H, gm);
        if (descending && gall<G>(mask == prev, gm)) break;  // nu is the root of this line
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
        float nn = (D - A) / H;
        if (alpha > 0.f && nn > 0.f) {
            const float tn = __logf(nn);
            if (tn > tcap) nn = slack_root(A, H, logbeta, alpha, tcap, tn, nu);
        }
        if (descending && !(nn < nu)) break;  // rounding: no further descent
        nu = nn;
        prev = mask;
        descending = true;
    }
    return nu;
}

// Bulk prefetch of [p, p + bytes) into L2 by the TMA engine (p and bytes
// multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One block (32/G demands, G lanes each): gather, x-block, scatter.
template <typename IdT, int KL, int G>
__device__ __forceinline__ void process_block(const IterArgs& a, int b, int lane, const float* __restrict__ xin,
                                              float* __restrict__ xout, const float* w_s,
                                              unsigned long long* h_s,
                                              float inv_beta, float logbeta, float beta_f, float alpha,
                                              KSum& ds2, KSum& x2, KSum& ex2) {
    const IdT* __restrict__ ids = static_cast<const IdT*>(a.L.ids);
    const IdT sentinel = (IdT)a.L.E;
    const unsigned gm = G == 1 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    // block metadata in one coalesced load: slot bases, then row offsets
    int sb = 0;
    if (lane < 2) sb = __ldg(&a.L.slotbase[b + lane]);
    const int s0 = __shfl_sync(0xffffffffu, sb, 0);
    const int KB = __shfl_sync(0xffffffffu, sb, 1) - s0;
    unsigned ro = 0u;
    if (lane <= KB) ro = __ldg(&a.L.rowoff[s0 + lane]);
    const size_t li = (size_t)b * kLanes + lane;
    const float D = __ldg(&a.L.Dn[li]);
    const float lam0 = __ldcg(&a.lam[li]);
    float xo[KL], m[KL], an[KL];
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        xo[j] = 0.f;
        if (j < KB) xo[j] = __ldcg(&xin[(size_t)(s0 + j) * kLanes + lane]);
    }
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        m[j] = 0.f; an[j] = 0.f;
        if (j < KB) {
            const unsigned r0 = __shfl_sync(0xffffffffu, ro, j), r1 = __shfl_sync(0xffffffffu, ro, j + 1);
            float q = 0.f;
            int n = 0;
            #pragma unroll 4
            for (unsigned r = r0; r < r1; ++r) {
                const IdT id = __ldg(&ids[(size_t)r * kLanes + lane]);
                q += w_s[id];
                n += (id != sentinel);
            }
            if (n > 0) {
                an[j] = __frcp_rn((float)n);
                m[j] = fmaf(-q, an[j], xo[j]);
            }
        }
    }
    float nu = 0.f;
    if (D > 0.f) {
        nu = solve_nu<KL, G>(m, an, D, inv_beta, logbeta, alpha, lam0 * inv_beta, gm);
        __stcg(&a.lam[li], nu * beta_f);
    }
    float bd = 0.f, bx = 0.f, be = 0.f;
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        if (j < KB) {
            const size_t sl = (size_t)(s0 + j);
            const float xn = an[j] > 0.f ? fmaxf(0.f, fmaf(nu, an[j], m[j])) : 0.f;
            __stcg(&xout[sl * kLanes + lane], xn);
            const float dx = xn - xo[j];
            bd = fmaf(dx, dx, bd);
            bx = fmaf(xn, xn, bx);
            const unsigned r0 = __shfl_sync(0xffffffffu, ro, j), r1 = __shfl_sync(0xffffffffu, ro, j + 1);
            if (xn != 0.f) {
                be = fmaf(xn * xn, __frcp_rn(an[j]), be);
                const unsigned long long fx = __float2ull_rn(xn * 0x1p32f);
                #pragma unroll 4
                for (unsigned r = r0; r < r1; ++r) {
                    const IdT id = __ldg(&ids[(size_t)r * kLanes + lane]);
                    if (id != sentinel) atomicAdd(&h_s[id], fx);
                }
            }
        }
    }
    ds2.add(bd);
    x2.add(bx);
    ex2.add(be);
}

// Distance, in blocks, of the rolling L2 prefetch window ahead of the
// blocks being processed by a CTA.
constexpr int kPrefetchAhead = 2 * kIterWarps;

template <typename IdT, int KL, int G>
__global__ void __launch_bounds__(kIterThreads, 1) k_iter(IterArgs a) {
    extern __shared__ __align__(16) unsigned long long smem[];
    const int E = a.L.E;
    // this CTA's edge-load histogram in 64-bit fixed point (2^-32 units):
    // integer atomics on shared memory are native, float ones are not
    unsigned long long* h_s = smem;                  // [E+1]
    float* w_s = reinterpret_cast<float*>(h_s + (E + 1));  // [E+1] gather weights u_e + d_e; w_s[E] = 0
    float* u_s = w_s + (E + 1);                      // [E]   scaled prices
    __shared__ double red[kIterWarps];
    __shared__ double s_fin[4];
    __shared__ int s_next;  // next block of this CTA's range (relative)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NG = gridDim.x;  // CTAs in the grid
    const int b_lo = a.cta_blk[blockIdx.x], b_hi = a.cta_blk[blockIdx.x + 1];
    if (tid == 0) s_next = 0;

    for (int e = tid; e < E; e += kIterThreads) {
        u_s[e] = a.u[e];
        w_s[e] = a.w[e];
        h_s[e] = 0ull;
    }
    if (tid == 0) { w_s[E] = 0.f; h_s[E] = 0ull; }
    Scalars sc = *a.sc;
    int xbuf = sc.xbuf;
    sc.converged = 0;
    sc.stop_reason = 0;
    __syncthreads();

    const size_t xstride = (size_t)a.L.nslots * kLanes;
    long long done = 0;
    (void)warp;

    for (long long it = 0; it < a.max_iters; ++it) {
        const float* __restrict__ xin = a.x + (size_t)xbuf * xstride;
        float* __restrict__ xout = a.x + (size_t)(xbuf ^ 1) * xstride;
        const float inv_beta = (float)(1.0 / sc.beta);
        const float logbeta = (float)log(sc.beta);
        const float beta_f = (float)sc.beta;
        const float alpha = (float)sc.alpha;
        KSum ds2, x2, ex2;

        // ---------------- phase A: per-demand rate updates ----------------
        // each CTA owns a contiguous range of blocks (balanced by their
        // rows); its warps take blocks one at a time from a shared counter.
        // The CTA's rows and rates are contiguous in memory, so the warp that
        // takes block b also prefetches block b + kPrefetchAhead into L2 (its
        // bounds are loaded when b is taken and the bulk prefetch is issued
        // after b is processed, so no warp waits on them).
        {
            const IdT* ids = static_cast<const IdT*>(a.L.ids);
            if (it == 0 && warp == 0) {
                // warm the start of the window
                const int pe = min(b_hi, b_lo + kPrefetchAhead);
                if (lane == 0 && pe > b_lo) {
                    const int s0 = __ldg(&a.L.slotbase[b_lo]), s1 = __ldg(&a.L.slotbase[pe]);
                    const unsigned r0 = __ldg(&a.L.rowoff[s0]), r1 = __ldg(&a.L.rowoff[s1]);
                    if (r1 > r0) prefetch_l2(ids + (size_t)r0 * kLanes, (unsigned)((r1 - r0) * kLanes * sizeof(IdT)));
                    if (s1 > s0) prefetch_l2(xin + (size_t)s0 * kLanes, (unsigned)((s1 - s0) * kLanes * sizeof(float)));
                }
            }
            while (true) {
                int b = 0;
                if (lane == 0) b = atomicAdd(&s_next, 1);
                b = __shfl_sync(0xffffffffu, b, 0) + b_lo;
                if (b >= b_hi) break;
                // bounds of the block kPrefetchAhead ahead (lanes 0-1 slot bases)
                const int bp = b + kPrefetchAhead;
                int psb = 0;
                if (bp < b_hi && lane < 2) psb = __ldg(&a.L.slotbase[bp + lane]);
                process_block<IdT, KL, G>(a, b, lane, xin, xout, w_s, h_s, inv_beta, logbeta, beta_f, alpha, ds2,
                                          x2, ex2);
                if (bp < b_hi) {
                    const int ps0 = __shfl_sync(0xffffffffu, psb, 0), ps1 = __shfl_sync(0xffffffffu, psb, 1);
                    unsigned pro = 0u;
                    if (lane < 2) pro = __ldg(&a.L.rowoff[lane == 0 ? ps0 : ps1]);
                    const unsigned pr0 = __shfl_sync(0xffffffffu, pro, 0), pr1 = __shfl_sync(0xffffffffu, pro, 1);
                    if (lane == 0) {
                        if (pr1 > pr0)
                            prefetch_l2(ids + (size_t)pr0 * kLanes, (unsigned)((pr1 - pr0) * kLanes * sizeof(IdT)));
                        if (ps1 > ps0)
                            prefetch_l2(xin + (size_t)ps0 * kLanes, (unsigned)((ps1 - ps0) * kLanes * sizeof(float)));
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_next = 0;
        // flush this CTA's loads into the global accumulator of this iteration
        float* Lg = a.loads + (size_t)(it % 3) * E;
        for (int e = tid; e < E; e += kIterThreads) {
            const unsigned long long v = h_s[e];
            if (v != 0ull) atomicAdd(&Lg[e], (float)((double)v * 0x1p-32));
            h_s[e] = 0ull;
        }
        {
            const double v0 = block_sum((double)ds2.s, red);
            const double v1 = block_sum((double)x2.s, red);
            const double v2 = block_sum((double)ex2.s, red);
            if (tid == 0) {
                double* p = a.part + ((size_t)(it & 1) * NG + blockIdx.x) * 4;
                __stcg(&p[0], v0);
                __stcg(&p[1], v1);
                __stcg(&p[2], v2);
            }
        }
        if (!grid_sync(a.barrier, (unsigned)((it + 1) * NG), a.status, a.timeout_ns,
                       (int)blockIdx.x != a.o.withhold_cta)) {
            break;
        }

        // ---------------- phase B: per-edge prices and control ----------------
        float rp = 0.f;
        {
            KSum r2;
            for (int e = tid; e < E; e += kIterThreads) {
                const float ne = __ldg(&a.L.ne_f[e]);
                const float u = u_s[e];
                float un = 0.f;
                if (ne > 0.f)
                    un = fmaxf(0.f, fmaf(__ldcg(&Lg[e]) - __ldg(&a.L.cap_n[e]), __ldg(&a.L.inv_ne[e]), u));
                const float d = un - u;
                r2.add(ne * d * d);
                u_s[e] = un;
                w_s[e] = un + d;
            }
            rp = r2.s;
        }
        const double r2s = block_sum((double)rp, red);
        if (tid < 32) {
            double v0 = 0.0, v1 = 0.0, v2 = 0.0;
            const double* p = a.part + (size_t)(it & 1) * NG * 4;
            for (int c = lane; c < NG; c += 32) {
                v0 += __ldcg(&p[c * 4 + 0]);
                v1 += __ldcg(&p[c * 4 + 1]);
                v2 += __ldcg(&p[c * 4 + 2]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            }
            if (lane == 0) { s_fin[0] = v0; s_fin[1] = v1; s_fin[2] = v2; }
        }
        __syncthreads();
        const double s_res = sqrt(s_fin[0]) / fmax(sqrt(s_fin[1]), 1e-30);
        const double r_res = sqrt(r2s) / fmax(sqrt(s_fin[2]), 1e-30);
        xbuf ^= 1;
        sc.iter_total++;
        sc.iter_alpha++;
        done++;
        int event = 0;
        if (!isfinite(s_res) || !isfinite(r_res)) {
            if (tid == 0 && blockIdx.x == 0) atomicCAS(a.status, 0, kStatusNumeric);
            sc.r = r_res;
            sc.s = s_res;
            break;
        }
        if (a.o.adapt_beta) {
            double nb = sc.beta;
            if (r_res > a.o.A * s_res) nb = sc.beta * a.o.C;
            else if (s_res > a.o.A * r_res) nb = sc.beta / a.o.C;
            if (nb != sc.beta) {
                const float ratio = (float)(sc.beta / nb);
                for (int e = tid; e < E; e += kIterThreads) {
                    const float u = u_s[e];
                    w_s[e] = fmaf(u, ratio - 1.f, w_s[e]);
                    u_s[e] = u * ratio;
                }
                sc.beta = nb;
                event |= 1;
            }
        }
        bool stop = false;
        if (r_res <= a.o.gamma && s_res <= a.o.gamma) {
            if (sc.alpha >= a.o.alpha_target) {
                stop = true; event |= 4;
            } else if (a.o.continuation && sc.iter_alpha == 1 && sc.alpha > a.o.alpha_start) {
                stop = true; event |= 8;
            } else if (sc.alpha >= a.o.alpha_max) {
                stop = true; event |= 16;
            } else {
                double na = sc.alpha + a.o.alpha_step;
                if (na > a.o.alpha_target) na = a.o.alpha_target;
                if (na > a.o.alpha_max) na = a.o.alpha_max;
                sc.alpha = na;
                sc.iter_alpha = 0;
                event |= 2;
            }
        }
        sc.r = r_res;
        sc.s = s_res;
        if (blockIdx.x == 0) {
            if (tid == 0 && a.trace_cap > 0) {
                double* t = a.trace + (size_t)((sc.iter_total - 1) % a.trace_cap) * kTraceWidth;
                t[0] = r_res; t[1] = s_res; t[2] = sc.beta; t[3] = sc.alpha; t[4] = (double)event;
            }
            // the load buffer used two iterations from now must start at zero
            float* Lz = a.loads + (size_t)((it + 2) % 3) * E;
            for (int e = tid; e < E; e += kIterThreads) __stcg(&Lz[e], 0.f);
        }
        __syncthreads();
        if (stop) {
            sc.converged = 1;
            sc.stop_reason = event & 28;
            break;
        }
    }
    if (blockIdx.x == 0) {
        for (int e = tid; e < E; e += kIterThreads) {
            a.u[e] = u_s[e];
            a.w[e] = w_s[e];
        }
        if (tid == 0) {
            sc.iters_run = done;
            sc.xbuf = xbuf;
            *a.sc = sc;
        }
    }
}

// Initial rates of Algorithm 1: x_r = D_c / |P_c| on every path of demand c
// (normalised units), 0 on padding slots.  One thread per lane; path p of a
// demand sits on lane t*G + p%G in slot p/G.
__global__ void k_init_x(Layout L, float* x) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * kLanes) return;
    const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
    const int hh = lane % L.G;
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    const int np = L.np[i];
    const float v = np > 0 ? L.Dn[i] / (float)np : 0.f;
    for (int j = 0; j < KB; ++j) x[(size_t)(s0 + j) * kLanes + lane] = j * L.G + hh < np ? v : 0.f;
}

template <typename IdT, int KL, int G>
cudaError_t launch_iter_t(const IterArgs& a, int grid, cudaStream_t st) {
    const size_t smem = iter_smem_bytes(a.L.E);
    cudaError_t err = cudaFuncSetAttribute(k_iter<IdT, KL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    IterArgs args = a;
    void* params[] = {&args};
    return cudaLaunchCooperativeKernel((const void*)k_iter<IdT, KL, G>, dim3(grid), dim3(kIterThreads), params,
                                       smem, st);
}

template <typename IdT, int KL, int G>
cudaError_t occupancy_t(int E, int* blocks) {
    const size_t smem = iter_smem_bytes(E);
    cudaError_t err = cudaFuncSetAttribute(k_iter<IdT, KL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_iter<IdT, KL, G>, kIterThreads, smem);
}

}  // namespace
}  // namespace te

namespace te {

size_t iter_smem_bytes(int E) {
    return (size_t)(E + 1) * sizeof(unsigned long long) + (size_t)(2 * (size_t)E + 1) * sizeof(float);
}

// instantiations: (paths per lane, lanes per demand) = (4,1), (8,1), (8,2), (8,4)
#define TE_DISPATCH(ID_BYTES, KL, G, CALL)                                       \
    do {                                                                         \
        if ((ID_BYTES) == 2) {                                                   \
            if ((G) == 1) return (KL) <= 4 ? CALL(uint16_t, 4, 1) : CALL(uint16_t, 8, 1); \
            if ((G) == 2) return CALL(uint16_t, 8, 2);                           \
            return CALL(uint16_t, 8, 4);                                         \
        }                                                                        \
        if ((G) == 1) return (KL) <= 4 ? CALL(int32_t, 4, 1) : CALL(int32_t, 8, 1); \
        if ((G) == 2) return CALL(int32_t, 8, 2);                                \
        return CALL(int32_t, 8, 4);                                              \
    } while (0)

cudaError_t iter_occupancy(int id_bytes, int kl, int G, int E, int* blocks_per_sm) {
#define TE_OCC(T, K, GG) occupancy_t<T, K, GG>(E, blocks_per_sm)
    TE_DISPATCH(id_bytes, kl, G, TE_OCC);
#undef TE_OCC
}

cudaError_t launch_iter(const IterArgs& a, int grid, cudaStream_t st) {
#define TE_LAUNCH(T, K, GG) launch_iter_t<T, K, GG>(a, grid, st)
    TE_DISPATCH(a.L.id_bytes, a.L.kl, a.L.G, TE_LAUNCH);
#undef TE_LAUNCH
}

cudaError_t launch_init_x(const Layout& L, float* x, cudaStream_t st) {
    const long long n = (long long)L.nblocks * kLanes;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    k_init_x<<<(unsigned)blocks, threads, 0, st>>>(L, x);
    return cudaGetLastError();
}

}  // namespace te

// Persistent iteration kernel of the GATE ADMM loop (Algorithm 1).
//
// One cooperative launch runs many iterations.  Per iteration:
//   phase A (every CTA, one warp per block of 32/G demands, G lanes per
//            demand): gather the consensus term of each path from the edge
//            weights w_e = u_e + d_e held in shared memory, solve the demand's
//            x-block (Eq. 14 and the sum computation of Appendix B.2), write
//            the new rates, and add each path's new rate into the CTA's
//            shared-memory histogram of edge loads (split 32-bit fixed point,
//            native shared-memory integer atomics).  The
//            edge ids of a block are brought into shared memory by one bulk
//            asynchronous copy (TMA), issued one block ahead of use; the
//            block's metadata record is loaded two blocks ahead.  The CTA then
//            publishes its per-edge partial loads and its FP64 residual
//            partials;
//   grid barrier 1;
//   phase B (every CTA, its own slice of the edges): the loads L_e as FP64
//            sums of the CTAs' partials in a fixed order (so a run is
//            deterministic), the per-edge price update
//            u_e' = max(0, u_e + (L_e - C_e)/n_e) (Eqs. 9/13 after the per-edge
//            collapse of the consensus duals) and its part of the primal
//            residual; publishes the new gather weights;
//   grid barrier 2;
//   control (every CTA, identically): the residuals r and s (Eqs. 15-16,
//            cross-CTA sums in FP64 in a fixed order), residual balancing
//            (Eq. 17), the stop rule (Eq. 18) and alpha-continuation, then
//            loads the new gather weights into shared memory.
// Every wait (grid barriers, bulk copies) is bounded.
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
            // the step only has to move t towards the root: its quotients
            // may be approximate (the accepted t still solves g(t) = 0)
            const float dg = __fdividef(H * et, s) + ia;
            tn = t - __fdividef(g, dg);
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
        float nn = (D - A) / H;
        if (nn > nucap) nn = slack_root(A, H, logbeta, alpha, tcap, __logf(nn), nu);
        if (descending && !(nn < nu)) break;  // rounding: no further descent
        nu = nn;
        prev = mask;
        descending = true;
    }
    return nu;
}


// ---------------------------------------------------------------------------
// bulk asynchronous copies and mbarriers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16), completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity; false on timeout.
__device__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
    }
    return true;
}

template <bool STAGED>
__device__ __forceinline__ uint16_t load_id(const uint16_t* p) {
    if (STAGED) {  // an explicit shared-memory load (the staging pointer is generic)
        unsigned short v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(smem_u32(p)));
        return v;
    }
    return __ldg(p);
}

// One block (32/G demands, G lanes each, at most 4 paths per lane): gather,
// x-block, scatter.  bids points at the block's first id row, in shared
// memory (STAGED) or in global memory.
// Per-lane inputs of one block read from global memory: the lane's rates,
// its demand and the demand's multiplier.  Loaded one block ahead of use.
struct BlockIn {
    float x[kMaxPathsPerLane];
    float D, lam;
};

template <int G>
__device__ __forceinline__ BlockIn load_block_in(const IterArgs& a, int b, int lane, int s0, int KB,
                                                 const float* __restrict__ xin) {
    BlockIn in;
    const size_t di = (size_t)b * a.L.dpb + lane / G;
    in.D = __ldg(&a.L.Dn[di]);
    in.lam = __ldcg(&a.lam[di]);
    #pragma unroll
    for (int j = 0; j < kMaxPathsPerLane; ++j) {
        in.x[j] = 0.f;
        if (j < KB) in.x[j] = __ldcg(&xin[(size_t)(s0 + j) * kLanes + lane]);
    }
    return in;
}

template <int G, bool STAGED>
__device__ __forceinline__ void process_block(const IterArgs& a, int b, int lane, const uint16_t* bids, int s0,
                                              unsigned counts, int KB, const BlockIn& in,
                                              float* __restrict__ xout, const float* w_s, unsigned* h_hi,
                                              unsigned* h_lo, float inv_beta, float logbeta,
                                              float beta_f, float alpha) {
    constexpr int KL = kMaxPathsPerLane;
    const uint16_t sentinel = (uint16_t)a.L.E;
    const unsigned gm = G == 1 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const size_t di = (size_t)b * a.L.dpb + lane / G;
    const float D = in.D;
    const float lam0 = in.lam;
    float xo[KL], m[KL], an[KL];
    #pragma unroll
    for (int j = 0; j < KL; ++j) xo[j] = in.x[j];
    unsigned rs = 0;  // first row of slot j within the block
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        m[j] = 0.f;
        an[j] = 0.f;
        if (j < KB) {
            const unsigned cnt = (counts >> (8 * j)) & 0xffu;
            float q = 0.f;
            int n = 0;
            #pragma unroll 4
            for (unsigned r = 0; r < cnt; ++r) {
                const uint16_t id = load_id<STAGED>(&bids[(size_t)(rs + r) * kLanes + lane]);
                q += w_s[id];
                n += (id != sentinel);
            }
            if (n > 0) {
                an[j] = __frcp_rn((float)n);
                m[j] = fmaf(-q, an[j], xo[j]);
            }
            rs += cnt;
        }
    }
    float nu = 0.f;
    if (D > 0.f) {
        nu = solve_nu<KL, G>(m, an, D, inv_beta, logbeta, alpha, lam0 * inv_beta, gm);
        if ((lane & (G - 1)) == 0) __stcg(&a.lam[di], nu * beta_f);
    }
    float bd = 0.f, bx = 0.f, be = 0.f;
    rs = 0;
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        if (j < KB) {
            const unsigned cnt = (counts >> (8 * j)) & 0xffu;
            const size_t sl = (size_t)(s0 + j);
            const float xn = an[j] > 0.f ? fmaxf(0.f, fmaf(nu, an[j], m[j])) : 0.f;
            __stcg(&xout[sl * kLanes + lane], xn);
            const float dx = xn - xo[j];
            bd = fmaf(dx, dx, bd);
            bx = fmaf(xn, xn, bx);
            if (xn != 0.f) {
                be = fmaf(xn * xn, __frcp_rn(an[j]), be);
                // split fixed point: integer part of xn * 2^12 and the
                // remaining fraction in units of 2^-24 (both exact in FP32)
                const float vf = xn * 0x1p12f;
                const float hf = floorf(vf);
                const unsigned hi = (unsigned)hf;
                const unsigned lo = (unsigned)__float2uint_rn((vf - hf) * 0x1p12f);
                // no per-row branch: padding entries (the sentinel id E) add
                // into the unused histogram slot E
                #pragma unroll 4
                for (unsigned r = 0; r < cnt; ++r) {
                    const uint16_t id = load_id<STAGED>(&bids[(size_t)(rs + r) * kLanes + lane]);
                    atomicAdd(&h_hi[id], hi);
                    atomicAdd(&h_lo[id], lo);
                }
            }
            rs += cnt;
        }
    }
    // the block's residual terms, summed over the warp in a fixed order and
    // stored per block, so that their totals do not depend on which warp
    // processed which block
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

__device__ __forceinline__ unsigned rows_of(unsigned counts) {
    return (counts & 0xffu) + ((counts >> 8) & 0xffu) + ((counts >> 16) & 0xffu) + (counts >> 24);
}

template <int G>
__global__ void __launch_bounds__(kIterThreads, 1) k_iter(IterArgs a) {
    extern __shared__ __align__(128) unsigned smem[];
    const int E = a.L.E;
    const int NG = gridDim.x;  // CTAs in the grid
    // dynamic shared memory: histogram, gather weights, staging, price slice
    unsigned* h_hi = smem;                                           // [E+1] units of 2^-12
    unsigned* h_lo = h_hi + (E + 1);                                 // [E+1] units of 2^-24
    float* w_s = reinterpret_cast<float*>(h_lo + (E + 1));          // [E+1], w_s[E] = 0
    uint16_t* stage = reinterpret_cast<uint16_t*>(
        reinterpret_cast<uintptr_t>(w_s + (E + 1) + 31) & ~uintptr_t(127));  // [warps][2][kStageRows*32]
    float* s_u = reinterpret_cast<float*>(stage + (size_t)kIterWarps * 2 * kStageRows * kLanes);  // price slice
    const int e_lo = (int)((long long)blockIdx.x * E / NG), e_hi = (int)((long long)(blockIdx.x + 1) * E / NG);
    float* s_un = s_u + (e_hi - e_lo);                               // next prices of the slice
    __shared__ __align__(8) unsigned long long s_mbar[kIterWarps * 2];
    __shared__ double red[kIterWarps];
    __shared__ double s_fin[4];
    __shared__ int s_next;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // blocks of this CTA: blockIdx.x, blockIdx.x + NG, ... (round robin, so
    // that every CTA gets a sample of all kinds of blocks)
    const int b_hi = a.L.nblocks;  // block indices >= b_hi mean "none"
    const int nbc = blockIdx.x < (unsigned)b_hi ? (b_hi - (int)blockIdx.x + NG - 1) / NG : 0;
    const uint16_t* ids = static_cast<const uint16_t*>(a.L.ids);
    uint16_t* wstage[2] = {stage + (size_t)(warp * 2) * kStageRows * kLanes,
                           stage + (size_t)(warp * 2 + 1) * kStageRows * kLanes};
    unsigned long long* mb = &s_mbar[warp * 2];

    for (int e = tid; e < E; e += kIterThreads) {
        w_s[e] = a.w[e];
        h_hi[e] = 0u;
        h_lo[e] = 0u;
    }
    for (int e = e_lo + tid; e < e_hi; e += kIterThreads) s_u[e - e_lo] = a.u[e];
    if (tid == 0) {
        w_s[E] = 0.f;
        h_hi[E] = 0u;
        h_lo[E] = 0u;
        s_next = 0;
    }
    if (lane == 0) {
        mbar_init(&mb[0], 1);
        mbar_init(&mb[1], 1);
        fence_mbar_init();
    }
    Scalars sc = *a.sc;
    int xbuf = sc.xbuf;
    sc.converged = 0;
    sc.stop_reason = 0;
    unsigned par[2] = {0u, 0u};  // phase parity of each staging buffer's mbarrier
    bool pending[2] = {false, false};
    bool failed = false;
    __syncthreads();

    const size_t xstride = (size_t)a.L.nslots * kLanes;
    long long done = 0;

    for (long long it = 0; it < a.max_iters; ++it) {
        const float* __restrict__ xin = a.x + (size_t)xbuf * xstride;
        float* __restrict__ xout = a.x + (size_t)(xbuf ^ 1) * xstride;
        const float inv_beta = (float)(1.0 / sc.beta);
        const float logbeta = (float)log(sc.beta);
        const float beta_f = (float)sc.beta;
        const float alpha = (float)sc.alpha;

        // ---------------- phase A: per-demand rate updates ----------------
        // Warps take the blocks of this CTA one at a time from a shared
        // counter (results do not depend on which warp takes which block:
        // the loads are integer sums and the residual terms are stored per
        // block).
        // The metadata record of the block after next is loaded (by lane 0),
        // and the next block's rates, demands and multipliers are loaded into
        // registers, while the bulk copy of the next block's ids runs and the
        // current block is processed.
        {
            auto grab = [&]() -> int {
                int v = 0;
                if (lane == 0) v = atomicAdd(&s_next, 1);
                v = __shfl_sync(0xffffffffu, v, 0);
                return v < nbc ? (int)blockIdx.x + v * NG : b_hi;
            };
            auto load_meta = [&](int b) -> BlockMeta {
                BlockMeta m{0u, 0u, 0u, 0u};
                if (lane == 0 && b < b_hi) m = a.L.blkmeta[b];
                return m;
            };
            // issues the bulk copy of block b into buffer k; returns whether
            // the block fits a staging buffer (else it is read from global)
            auto issue = [&](int b, const BlockMeta& m, int k) -> bool {
                const unsigned counts = __shfl_sync(0xffffffffu, m.counts, 0);
                const unsigned row0 = __shfl_sync(0xffffffffu, m.row0, 0);
                const unsigned rows = rows_of(counts);
                if (rows > (unsigned)kStageRows || rows == 0) return false;
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async_smem();
                    const unsigned bytes = rows * kLanes * (unsigned)sizeof(uint16_t);
                    mbar_expect_tx(&mb[k], bytes);
                    bulk_g2s(wstage[k], ids + (size_t)row0 * kLanes, bytes, &mb[k]);
                }
                pending[k] = true;
                (void)b;
                return true;
            };
            auto prefetch = [&](int b, const BlockMeta& m) -> BlockIn {
                const int s0 = (int)__shfl_sync(0xffffffffu, m.s0, 0);
                const int KB = (int)__shfl_sync(0xffffffffu, m.kb, 0);
                BlockIn in{};
                if (b < b_hi) in = load_block_in<G>(a, b, lane, s0, KB, xin);
                return in;
            };
            int b0 = grab();
            BlockMeta m0 = load_meta(b0);
            int b1 = grab();
            BlockMeta m1 = load_meta(b1);
            int cur = 0;
            bool st0 = (b0 < b_hi) && !failed ? issue(b0, m0, cur) : false;
            BlockIn in0 = prefetch(b0, m0);
            while (b0 < b_hi && !failed) {
                const int b2 = grab();
                const BlockMeta m2 = load_meta(b2);
                const bool st1 = (b1 < b_hi) ? issue(b1, m1, cur ^ 1) : false;
                const BlockIn in1 = prefetch(b1, m1);
                const int s0 = (int)__shfl_sync(0xffffffffu, m0.s0, 0);
                const unsigned counts = __shfl_sync(0xffffffffu, m0.counts, 0);
                const int KB = (int)__shfl_sync(0xffffffffu, m0.kb, 0);
                if (st0) {
                    if (!mbar_wait(&mb[cur], par[cur], a.timeout_ns)) {
                        if (lane == 0) atomicCAS(a.status, 0, kStatusTimeout);
                        failed = true;
                        break;
                    }
                    par[cur] ^= 1u;
                    pending[cur] = false;
                    process_block<G, true>(a, b0, lane, wstage[cur], s0, counts, KB, in0, xout, w_s, h_hi, h_lo,
                                           inv_beta, logbeta, beta_f, alpha);
                } else {
                    const unsigned row0 = __shfl_sync(0xffffffffu, m0.row0, 0);
                    process_block<G, false>(a, b0, lane, ids + (size_t)row0 * kLanes, s0, counts, KB, in0, xout,
                                            w_s, h_hi, h_lo, inv_beta, logbeta, beta_f, alpha);
                }
                b0 = b1;
                m0 = m1;
                in0 = in1;
                st0 = st1;
                b1 = b2;
                m1 = m2;
                cur ^= 1;
            }
        }
        __syncthreads();
        if (tid == 0) s_next = 0;  // read again only after the next barriers
        // publish this CTA's partial loads
        uint2* Lp = a.loads + (size_t)blockIdx.x * E;
        for (int e = tid; e < E; e += kIterThreads) {
            __stcg(&Lp[e], make_uint2(h_hi[e], h_lo[e]));
            h_hi[e] = 0u;
            h_lo[e] = 0u;
        }
        {
            // this CTA's residual partials: its blocks' terms in FP64, each
            // thread over a fixed stride of the block range, then a fixed-order
            // CTA reduction
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int k = tid; k < nbc; k += kIterThreads) {
                const float* r = a.blkres + ((size_t)blockIdx.x + (size_t)k * NG) * 3;
                t0 += (double)__ldcg(&r[0]);
                t1 += (double)__ldcg(&r[1]);
                t2 += (double)__ldcg(&r[2]);
            }
            const double v0 = block_sum(t0, red);
            const double v1 = block_sum(t1, red);
            const double v2 = block_sum(t2, red);
            if (tid == 0) {
                double* p = a.part + ((size_t)(it & 1) * NG + blockIdx.x) * 4;
                __stcg(&p[0], v0);
                __stcg(&p[1], v1);
                __stcg(&p[2], v2);
            }
        }
        if (!grid_sync(a.barrier, (unsigned)((2 * it + 1) * NG), a.status, a.timeout_ns,
                       (int)blockIdx.x != a.o.withhold_cta)) {
            failed = true;
            break;
        }

        // ---------------- phase B: this CTA's slice of the edge prices ----------------
        {
            // L_e of the slice: the CTAs' integer partials summed exactly in
            // 64 bits (so L_e does not depend on how blocks are spread over
            // CTAs) and converted once; thread t adds the partials of CTAs
            // c = t / ns, t / ns + kIterThreads / ns, ... for edge e_lo + t % ns
            const int ns = e_hi - e_lo;
            unsigned long long* s_L = reinterpret_cast<unsigned long long*>(
                (reinterpret_cast<uintptr_t>(s_un + ns) + 7) & ~uintptr_t(7));  // [2][kIterThreads]
            if (ns > 0) {
                const int per = kIterThreads / ns > 0 ? kIterThreads / ns : 1;
                unsigned long long sh = 0ull, sl = 0ull;
                if (tid < per * ns) {
                    const int e = e_lo + tid % ns;
                    for (int c = tid / ns; c < NG; c += per) {
                        const uint2 v = __ldcg(&a.loads[(size_t)c * E + e]);
                        sh += v.x;
                        sl += v.y;
                    }
                }
                s_L[tid] = sh;
                s_L[kIterThreads + tid] = sl;
                __syncthreads();
                if (tid < ns) {
                    unsigned long long H = 0ull, Lo = 0ull;
                    for (int k = 0; k < per; ++k) {
                        H += s_L[k * ns + tid];
                        Lo += s_L[kIterThreads + k * ns + tid];
                    }
                    s_L[tid] = H;  // each slot read and written by its own thread only
                    s_L[kIterThreads + tid] = Lo;
                }
                __syncthreads();
            }
            KSum r2;
            for (int e = e_lo + tid; e < e_hi; e += kIterThreads) {
                const float ne = __ldg(&a.L.ne_f[e]);
                const float u = s_u[e - e_lo];
                const float L = (float)((double)s_L[e - e_lo] * 0x1p-12 + (double)s_L[kIterThreads + e - e_lo] * 0x1p-24);
                float un = 0.f;
                if (ne > 0.f) un = fmaxf(0.f, fmaf(L - __ldg(&a.L.cap_n[e]), __ldg(&a.L.inv_ne[e]), u));
                const float d = un - u;
                r2.add(ne * d * d);
                s_un[e - e_lo] = un;
                __stcg(&a.u_next[e], un);
                __stcg(&a.w_next[e], un + d);
            }
            const double v3 = block_sum((double)r2.s, red);
            if (tid == 0) __stcg(&a.part[((size_t)(it & 1) * NG + blockIdx.x) * 4 + 3], v3);
        }
        if (!grid_sync(a.barrier, (unsigned)((2 * it + 2) * NG), a.status, a.timeout_ns, true)) {
            failed = true;
            break;
        }

        // ---------------- control: residuals, beta, alpha, stop ----------------
        if (tid < 32) {
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            const double* p = a.part + (size_t)(it & 1) * NG * 4;
            for (int c = lane; c < NG; c += 32) {
                v0 += __ldcg(&p[c * 4 + 0]);
                v1 += __ldcg(&p[c * 4 + 1]);
                v2 += __ldcg(&p[c * 4 + 2]);
                v3 += __ldcg(&p[c * 4 + 3]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                v3 += __shfl_xor_sync(0xffffffffu, v3, o);
            }
            if (lane == 0) { s_fin[0] = v0; s_fin[1] = v1; s_fin[2] = v2; s_fin[3] = v3; }
        }
        __syncthreads();
        const double s_res = sqrt(s_fin[0]) / fmax(sqrt(s_fin[1]), 1e-30);
        const double r_res = sqrt(s_fin[3]) / fmax(sqrt(s_fin[2]), 1e-30);
        xbuf ^= 1;
        sc.iter_total++;
        sc.iter_alpha++;
        done++;
        int event = 0;
        const bool numeric_ok = isfinite(s_res) && isfinite(r_res);
        float ratio = 1.f;
        if (numeric_ok && a.o.adapt_beta) {
            double nb = sc.beta;
            if (r_res > a.o.A * s_res) nb = sc.beta * a.o.C;
            else if (s_res > a.o.A * r_res) nb = sc.beta / a.o.C;
            if (nb != sc.beta) {
                ratio = (float)(sc.beta / nb);
                sc.beta = nb;
                event |= 1;
            }
        }
        // commit the slice's new prices (scaled with beta) and the new gather
        // weights w = u' + d (the rescale keeps d, a primal quantity)
        for (int e = e_lo + tid; e < e_hi; e += kIterThreads) s_u[e - e_lo] = s_un[e - e_lo] * ratio;
        for (int e = tid; e < E; e += kIterThreads) {
            float w = __ldcg(&a.w_next[e]);
            if (ratio != 1.f) w = fmaf(__ldcg(&a.u_next[e]), ratio - 1.f, w);
            w_s[e] = w;
        }
        if (!numeric_ok) {
            if (tid == 0 && blockIdx.x == 0) atomicCAS(a.status, 0, kStatusNumeric);
            sc.r = r_res;
            sc.s = s_res;
            __syncthreads();
            break;
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
        if (blockIdx.x == 0 && tid == 0 && a.trace_cap > 0) {
            double* t = a.trace + (size_t)((sc.iter_total - 1) % a.trace_cap) * kTraceWidth;
            t[0] = r_res; t[1] = s_res; t[2] = sc.beta; t[3] = sc.alpha; t[4] = (double)event;
        }
        __syncthreads();
        if (stop) {
            sc.converged = 1;
            sc.stop_reason = event & 28;
            break;
        }
    }
    // a warp that gave up may still have bulk copies in flight into its
    // staging buffers: wait for them (bounded) before the CTA exits
    if (failed) {
        for (int k = 0; k < 2; ++k)
            if (pending[k]) mbar_wait(&mb[k], par[k], a.timeout_ns);
    }
    __syncthreads();
    for (int e = e_lo + tid; e < e_hi; e += kIterThreads) a.u[e] = s_u[e - e_lo];
    if (blockIdx.x == 0) {
        for (int e = tid; e < E; e += kIterThreads) a.w[e] = w_s[e];
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
    const size_t di = (size_t)b * L.dpb + lane / L.G;
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    const int np = L.np[di];
    const float v = np > 0 ? L.Dn[di] / (float)np : 0.f;
    for (int j = 0; j < KB; ++j) x[(size_t)(s0 + j) * kLanes + lane] = j * L.G + hh < np ? v : 0.f;
}

template <int G>
cudaError_t launch_iter_t(const IterArgs& a, int grid, cudaStream_t st) {
    const size_t smem = iter_smem_bytes(a.L.E, grid);
    cudaError_t err = cudaFuncSetAttribute(k_iter<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    IterArgs args = a;
    void* params[] = {&args};
    return cudaLaunchCooperativeKernel((const void*)k_iter<G>, dim3(grid), dim3(kIterThreads), params, smem, st);
}

template <int G>
cudaError_t occupancy_t(int E, int grid_hint, int* blocks) {
    const size_t smem = iter_smem_bytes(E, grid_hint);
    cudaError_t err = cudaFuncSetAttribute(k_iter<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_iter<G>, kIterThreads, smem);
}

}  // namespace

// Dynamic shared memory of the iteration kernel: histogram (8 B per edge),
// gather weights (4 B per edge), staging buffers, and the CTA's price slice
// (current and next) for a grid of at least `grid` CTAs.
size_t iter_smem_bytes(int E, int grid) {
    size_t b = 2 * (size_t)(E + 1) * sizeof(unsigned) + (size_t)(E + 1) * sizeof(float);
    b = (b + 31 * sizeof(float) + 127) & ~size_t(127);
    b += (size_t)kIterWarps * 2 * kStageRows * kLanes * sizeof(uint16_t);
    const int slice = (E + grid - 1) / (grid > 0 ? grid : 1) + 1;
    b += 2 * (size_t)slice * sizeof(float);
    b = (b + 7) & ~size_t(7);
    b += 2 * (size_t)kIterThreads * sizeof(unsigned long long);
    return b;
}

cudaError_t iter_occupancy(int G, int E, int grid_hint, int* blocks_per_sm) {
    switch (G) {
        case 1: return occupancy_t<1>(E, grid_hint, blocks_per_sm);
        case 2: return occupancy_t<2>(E, grid_hint, blocks_per_sm);
        case 4: return occupancy_t<4>(E, grid_hint, blocks_per_sm);
        default: return occupancy_t<8>(E, grid_hint, blocks_per_sm);
    }
}

cudaError_t launch_iter(const IterArgs& a, int grid, cudaStream_t st) {
    switch (a.L.G) {
        case 1: return launch_iter_t<1>(a, grid, st);
        case 2: return launch_iter_t<2>(a, grid, st);
        case 4: return launch_iter_t<4>(a, grid, st);
        default: return launch_iter_t<8>(a, grid, st);
    }
}

cudaError_t launch_init_x(const Layout& L, float* x, cudaStream_t st) {
    const long long n = (long long)L.nblocks * kLanes;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    k_init_x<<<(unsigned)blocks, threads, 0, st>>>(L, x);
    return cudaGetLastError();
}

}  // namespace te

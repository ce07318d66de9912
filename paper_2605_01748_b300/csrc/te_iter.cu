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
//            edge ids of a block are brought into shared memory by 16-byte
//            asynchronous copies (cp.async), issued one block ahead of use; the
//            block's metadata record is loaded two blocks ahead.  The CTA then
//            publishes its per-edge partial loads and its residual partials
//            (each lane's sums over its warp's blocks compensated in FP32,
//            everything above the lane in FP64);
//   grid barrier 1;
//   phase B (every CTA, its own slice of the edges): the loads L_e as FP64
//            sums of the CTAs' partials in a fixed order (so a run is
//            deterministic), the per-edge price update
//            u_e' = max(0, u_e + (L_e - C_e)/n_e) (Eqs. 9/13 after the per-edge
//            collapse of the consensus duals) and its part of the primal
//            residual; publishes the new gather weights;
//   grid barrier 2;
//   control (every CTA, identically, on thread 0): the residuals r and s
//            (Eqs. 15-16, cross-CTA sums in FP64 in a fixed order), residual
//            balancing (Eq. 17), the stop rule (Eq. 18) and
//            alpha-continuation; the CTA then loads the new gather weights
//            into shared memory.
// Every wait on another CTA (the grid barriers) is bounded.
//
// Rates and prices are FP32.  The per-demand multiplier is kept in scaled
// form nu = lambda / beta, so x_r = max(0, m_r + nu / n_r) with
// m_r = x_r - (1/n_r) sum_{e in r} w_e, and lambda = U'(S) = S^-alpha becomes
// beta nu S^alpha = 1, solved in the log domain (no overflow of S^-alpha at
// large alpha).
#include <math.h>
#include <stdint.h>

#include "te_kernels.cuh"

namespace te {
namespace {

// DET: exact split fixed-point load histograms (two 32-bit integer atomics
// per incidence); else one FP32 histogram (one FP32 atomic per incidence).
// GROUPED: the grid runs several independent instances, `group` CTAs each:
// CTA c takes instance c / group, whose arguments it reads from group_args
// (each instance has its own barrier counter, scalars and scratch); else the
// whole grid runs the one instance of a_param.
// WIDE (with DET, not GROUPED): the wide-edge mode for instances whose
// per-edge arrays do not fit shared memory.  Each CTA keeps its gather
// weights (a.wpriv) and its load histogram (a.hist64: one 64-bit
// fixed-point word per edge, units of 2^-24, one 64-bit reduction per
// incidence into L2) in its own slice of global memory; phase B sums the
// CTAs' words exactly, so the loads, and the whole run, are bit-identical
// to the shared-memory mode on the same instance.
// IdT: the layout's edge id type; 32-bit ids (above 65,534 edges) only in
// the wide-edge mode, where the staging buffers take the room of the
// per-edge arrays.
// KL: path slots per lane (kMaxPathsPerLane, or 1 for layouts with one path
// per lane: the single-path demands of k = 1 instances).
template <int G, bool DET, bool GROUPED, bool WIDE = false, typename IdT = uint16_t, int KL = kMaxPathsPerLane>
__global__ void __launch_bounds__(kIterThreads, 1)
    k_iter(IterArgs a_param, const IterArgs* __restrict__ group_args, int group) {
    static_assert(!WIDE || (DET && !GROUPED), "the wide-edge mode has deterministic loads and one instance");
    static_assert(sizeof(IdT) == 2 || WIDE, "32-bit edge ids only in the wide-edge mode");
    constexpr size_t kIdHalves = sizeof(IdT) / sizeof(uint16_t);  // staging size in 16-bit units per id
    extern __shared__ __align__(128) unsigned smem[];
    __shared__ IterArgs s_args;
    if (GROUPED) {
        if (threadIdx.x == 0) s_args = group_args[blockIdx.x / group];
        __syncthreads();
    }
    const IterArgs& a = GROUPED ? s_args : a_param;
    const int E = a.L.E;
    const int NG = GROUPED ? group : (int)gridDim.x;  // CTAs of this instance
    const int cta = GROUPED ? (int)(blockIdx.x % group) : (int)blockIdx.x;  // this CTA's rank among them
    // dynamic shared memory: histogram, gather weights, staging, price slice
    // (WIDE: staging and price slice; histogram and weights in global memory)
    unsigned* h_hi = WIDE ? reinterpret_cast<unsigned*>(a.hist64 + (size_t)cta * (E + 1))
                          : smem;                                    // [E+1] units of 2^-12 (DET), else FP32
    unsigned long long* h64 = WIDE ? a.hist64 + (size_t)cta * (E + 1) : nullptr;  // [E+1] units of 2^-24 (WIDE)
    unsigned* h_lo = (DET && !WIDE) ? h_hi + (E + 1) : nullptr;      // [E+1] units of 2^-24 (DET)
    float* w_s = WIDE ? a.wpriv + (size_t)cta * (E + 1)
                      : reinterpret_cast<float*>(h_hi + (DET ? 2 : 1) * (E + 1));  // [E+1], w_s[E] = 0
    uint16_t* stage = WIDE ? reinterpret_cast<uint16_t*>(smem)
                           : reinterpret_cast<uint16_t*>(reinterpret_cast<uintptr_t>(w_s + (E + 1) + 31) &
                                                         ~uintptr_t(127));  // [warps][2][kIterStageRows*32]
    float* s_u = reinterpret_cast<float*>(stage + (size_t)kIterWarps * 2 * kIterStageRows * kLanes * kIdHalves);  // price slice
    const int e_lo = (int)((long long)cta * E / NG), e_hi = (int)((long long)(cta + 1) * E / NG);
    float* s_un = s_u + (e_hi - e_lo);                               // next prices of the slice
    __shared__ double s_wred[kIterWarps][4];  // per-warp FP64 partials of the residual sums
    __shared__ float s_wmax[kIterWarps];      // per-warp largest relative capacity violation
    __shared__ float s_par[5];   // this iteration's 1/beta, log beta, beta, alpha, 1/alpha (FP32)
    __shared__ float s_ratio;    // price rescale of the last balancing step
    __shared__ int s_ctl;        // control decision: bit 0 numeric failure, bit 1 stop

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // blocks of this CTA: cta, cta + NG, ... (round robin, so
    // that every CTA gets a sample of all kinds of blocks)
    const int b_hi = a.L.nblocks;  // block indices >= b_hi mean "none"
    const int nbc = cta < b_hi ? (b_hi - cta + NG - 1) / NG : 0;
    const IdT* ids = static_cast<const IdT*>(a.L.ids);
    WarpStage ws;
    ws.base = stage + (size_t)(warp * 2) * kIterStageRows * kLanes * kIdHalves;

    for (int e = tid; e < E; e += kIterThreads) {
        w_s[e] = a.w[e];
        if (WIDE) {
            h64[e] = 0ull;
        } else {
            h_hi[e] = 0u;  // also FP32 +0
            if (DET) h_lo[e] = 0u;
        }
    }
    for (int e = e_lo + tid; e < e_hi; e += kIterThreads) s_u[e - e_lo] = a.u[e];
    if (tid == 0) {
        w_s[E] = 0.f;
        if (WIDE) {
            h64[E] = 0ull;
        } else {
            h_hi[E] = 0u;
            if (DET) h_lo[E] = 0u;
        }
    }
    // the scalar state is kept by thread 0, which takes the control
    // decisions (FP64 is slow on this part: one thread does it and the CTA
    // reads the results from shared memory)
    Scalars sc = *a.sc;
    int xbuf = sc.xbuf;
    sc.converged = 0;
    sc.stop_reason = 0;
    bool failed = false;
    auto publish_params = [&]() {
        s_par[0] = (float)(1.0 / sc.beta);
        s_par[1] = (float)log(sc.beta);
        s_par[2] = (float)sc.beta;
        s_par[3] = (float)sc.alpha;
        s_par[4] = sc.alpha > 0.0 ? 1.f / (float)sc.alpha : 0.f;
    };
    if (tid == 0) publish_params();
    __syncthreads();

    const size_t xstride = a.xstride > 0 ? (size_t)a.xstride : (size_t)a.L.nslots * kLanes;
    long long done = 0;

    for (long long it = 0; it < a.max_iters; ++it) {
        const float* __restrict__ xin = a.x + (size_t)xbuf * xstride;
        float* __restrict__ xout = a.x + (size_t)(xbuf ^ 1) * xstride;
        const float inv_beta = s_par[0];
        const float logbeta = s_par[1];
        const float beta_f = s_par[2];
        const float alpha = s_par[3];
        const float inv_alpha = s_par[4];

        // ---------------- phase A: per-demand rate updates ----------------
        // The warps share the blocks of this CTA (cta, cta +
        // NG, ...) in a fixed interleave, so a run is deterministic (the
        // loads are integer sums, and each lane sums the residual terms of
        // its warp's blocks, compensated, in the order of the interleave).
        LaneRes acc;
        if (!failed) {
            const BlockCtx bc{a.L.Dn, a.lam, nullptr, a.L.hops, a.L.dpb, (uint16_t)a.L.E};
            run_blocks<G, kIterStageRows, true, true, DET, WIDE, IdT, KL>(cta, NG, nbc, a.L.blkmeta, ids, xin, xout, bc, ws,
                                                w_s, h_hi, h_lo, inv_beta, logbeta, beta_f, alpha, inv_alpha, acc);
        }
        {
            // this warp's residual partials: each lane's compensated sums in
            // FP64, summed over the warp in a fixed butterfly (done here, so
            // that warps that finish early do it while the others still run)
            double t0 = acc.d.value(), t1 = (double)acc.x, t2 = (double)acc.e;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
                t2 += __shfl_xor_sync(0xffffffffu, t2, o);
            }
            if (lane == 0) {
                s_wred[warp][0] = t0;
                s_wred[warp][1] = t1;
                s_wred[warp][2] = t2;
            }
        }
        __syncthreads();
        // publish this CTA's partial loads (WIDE: they are in global memory
        // already, and are cleared after the second grid barrier)
        if (WIDE) {
        } else if (DET) {
            uint2* Lp = a.loads + (size_t)cta * E;
            #pragma unroll 4
            for (int e = tid; e < E; e += kIterThreads) {
                __stcg(&Lp[e], make_uint2(h_hi[e], h_lo[e]));
                h_hi[e] = 0u;
                h_lo[e] = 0u;
            }
        } else {
            float* Lp = reinterpret_cast<float*>(a.loads) + (size_t)cta * E;
            const float* hf = reinterpret_cast<const float*>(h_hi);
            #pragma unroll 4
            for (int e = tid; e < E; e += kIterThreads) {
                __stcg(&Lp[e], hf[e]);
                h_hi[e] = 0u;
            }
        }
        {
            // this CTA's residual partials: the warps' sums added in warp
            // order by thread 0 (the blocks of a warp are fixed by the
            // interleave, so the totals do not depend on timing)
            if (tid == 0) {
                double v0 = 0.0, v1 = 0.0, v2 = 0.0;
                for (int w = 0; w < kIterWarps; ++w) {
                    v0 += s_wred[w][0];
                    v1 += s_wred[w][1];
                    v2 += s_wred[w][2];
                }
                double* p = a.part + ((size_t)(it & 1) * NG + cta) * kPartWidth;
                __stcg(&p[0], v0);
                __stcg(&p[1], v1);
                __stcg(&p[2], v2);
            }
        }
        if (!grid_sync(a.barrier, (unsigned)((2 * it + 1) * NG), a.status, a.timeout_ns,
                       cta != a.o.withhold_cta)) {
            failed = true;
            break;
        }

        // ---------------- phase B: this CTA's slice of the edge prices ----------------
        {
            // L_e of the slice, in chunks of at most kIterThreads edges: the
            // CTAs' integer partials summed exactly in 64 bits (DET: so L_e
            // does not depend on how blocks are spread over CTAs) and
            // converted once, or the CTAs' FP32 partials summed in FP64 in CTA
            // order; thread t adds the partials of CTAs c = t / ns,
            // t / ns + kIterThreads / ns, ... for edge c0 + t % ns of the chunk
            // [2][kIterThreads] in the staging buffers, idle in phase B
            // (every copy of phase A has landed; the next are issued after
            // the control section's barrier)
            static_assert(2 * kIterThreads * sizeof(unsigned long long) <=
                              (size_t)kIterWarps * 2 * kIterStageRows * kLanes * sizeof(uint16_t),
                          "the phase-B partial sums fit the staging buffers");
            unsigned long long* s_L = reinterpret_cast<unsigned long long*>(stage);
            double* s_Ld = reinterpret_cast<double*>(stage);
            KSum r2;
            float vmax = 0.f;  // largest relative capacity violation n_e |d_e| / C_e of the slice
            for (int c0 = e_lo; c0 < e_hi; c0 += kIterThreads) {
                const int ns = min(kIterThreads, e_hi - c0);
                const int per = kIterThreads / ns;
                if (DET) {
                    unsigned long long sh = 0ull, sl = 0ull;
                    if (tid < per * ns) {
                        const int e = c0 + tid % ns;
                        // all of a thread's partials in flight at once (about NG /
                        // per of them: one L2 round trip instead of several)
                        if (WIDE) {
                            // the CTAs' words in units of 2^-24 (sh); sl stays 0
                            #pragma unroll 16
                            for (int c = tid / ns; c < NG; c += per) sh += __ldcg(&a.hist64[(size_t)c * (E + 1) + e]);
                        } else {
                            #pragma unroll 16
                            for (int c = tid / ns; c < NG; c += per) {
                                const uint2 v = __ldcg(&a.loads[(size_t)c * E + e]);
                                sh += v.x;
                                sl += v.y;
                            }
                        }
                    }
                    s_L[tid] = sh;
                    s_L[kIterThreads + tid] = sl;
                } else {
                    const float* Lf = reinterpret_cast<const float*>(a.loads);
                    double sf = 0.0;
                    if (tid < per * ns) {
                        const int e = c0 + tid % ns;
                        #pragma unroll 4
                        for (int c = tid / ns; c < NG; c += per) sf += (double)__ldcg(&Lf[(size_t)c * E + e]);
                    }
                    s_Ld[tid] = sf;
                }
                __syncthreads();
                if (tid < ns) {
                    if (DET) {
                        unsigned long long H = 0ull, Lo = 0ull;
                        for (int k = 0; k < per; ++k) {
                            H += s_L[k * ns + tid];
                            Lo += s_L[kIterThreads + k * ns + tid];
                        }
                        s_L[tid] = H;  // each slot read and written by its own thread only
                        s_L[kIterThreads + tid] = Lo;
                    } else {
                        double F = 0.0;
                        for (int k = 0; k < per; ++k) F += s_Ld[k * ns + tid];
                        s_Ld[tid] = F;
                    }
                }
                __syncthreads();
                if (tid < ns) {
                    const int e = c0 + tid;
                    const float ne = __ldg(&a.L.ne_f[e]);
                    const float u = s_u[e - e_lo];
                    // (WIDE: one exact sum in units of 2^-24; the same value as the
                    // split sum, both being the correctly rounded FP64 of the
                    // same integer multiple of 2^-24)
                    const float L = WIDE  ? (float)((double)s_L[tid] * 0x1p-24)
                                    : DET ? (float)((double)s_L[tid] * 0x1p-12 + (double)s_L[kIterThreads + tid] * 0x1p-24)
                                          : (float)s_Ld[tid];
                    float un = 0.f;
                    const float cap = __ldg(&a.L.cap_n[e]);
                    if (ne > 0.f) un = fmaxf(0.f, fmaf(L - cap, __ldg(&a.L.inv_ne[e]), u));
                    const float d = un - u;
                    r2.add(ne * d * d);
                    if (ne > 0.f) vmax = fmaxf(vmax, __fdiv_ru(ne * fabsf(d), cap));
                    s_un[e - e_lo] = un;
                    __stcg(&a.u_next[e], un);
                    __stcg(&a.w_next[e], un + d);
                }
                __syncthreads();  // the next chunk reuses s_L
            }
            double t3 = r2.value();
            if (warp * 32 < min(kIterThreads, e_hi - e_lo)) {  // the other warps hold no edge: 0
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    t3 += __shfl_xor_sync(0xffffffffu, t3, o);
                    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
                }
            }
            if (lane == 0) {
                s_wred[warp][3] = t3;
                s_wmax[warp] = vmax;
            }
            __syncthreads();
            if (tid == 0) {
                double v3 = 0.0;
                float m = 0.f;
                for (int w = 0; w < kIterWarps; ++w) {
                    v3 += s_wred[w][3];
                    m = fmaxf(m, s_wmax[w]);
                }
                double* p = a.part + ((size_t)(it & 1) * NG + cta) * kPartWidth;
                __stcg(&p[3], v3);
                __stcg(&p[4], (double)m);
            }
        }
        if (!grid_sync(a.barrier, (unsigned)((2 * it + 2) * NG), a.status, a.timeout_ns, true)) {
            failed = true;
            break;
        }

        // ---------------- control: residuals, beta, alpha, stop ----------------
        // warp 0 sums the CTAs' partials (FP64, fixed order, identical in
        // every CTA); thread 0 takes the decisions and publishes them
        xbuf ^= 1;
        done++;
        if (tid < 32) {
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0;
            const double* p = a.part + (size_t)(it & 1) * NG * kPartWidth;
            #pragma unroll 8  // a lane's loads in flight together (NG / 32 rounds of L2 latency otherwise)
            for (int c = lane; c < NG; c += 32) {
                v0 += __ldcg(&p[c * kPartWidth + 0]);
                v1 += __ldcg(&p[c * kPartWidth + 1]);
                v2 += __ldcg(&p[c * kPartWidth + 2]);
                v3 += __ldcg(&p[c * kPartWidth + 3]);
                v4 = fmax(v4, __ldcg(&p[c * kPartWidth + 4]));
            }
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                v3 += __shfl_xor_sync(0xffffffffu, v3, o);
                v4 = fmax(v4, __shfl_xor_sync(0xffffffffu, v4, o));
            }
            if (tid == 0) {
                const double s_res = sqrt(v0) / fmax(sqrt(v1), 1e-30);
                const double r_res = sqrt(v3) / fmax(sqrt(v2), 1e-30);
                sc.iter_total++;
                sc.iter_alpha++;
                int event = 0, ctl = 0;
                float ratio = 1.f;
                const bool numeric_ok = isfinite(s_res) && isfinite(r_res);
                if (numeric_ok && a.o.adapt_beta && fmax(r_res, s_res) > a.o.balance_floor) {
                    const double nb = balanced_beta(sc.beta, r_res, s_res, a.o.A, a.o.C, a.o.beta_cap);
                    if (nb != sc.beta) {
                        ratio = (float)(sc.beta / nb);
                        sc.beta = nb;
                        event |= 1;
                    }
                }
                if (!numeric_ok) {
                    ctl = 1;
                    if (cta == 0) atomicCAS(a.status, 0, kStatusNumeric);
                } else if (r_res <= a.o.gamma && s_res <= a.o.gamma && (a.o.gamma_max <= 0.0 || v4 <= a.o.gamma_max)) {
                    bool stop = false;
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
                    if (stop) {
                        ctl = 2;
                        sc.converged = 1;
                        sc.stop_reason = event & 28;
                    }
                }
                sc.r = r_res;
                sc.s = s_res;
                if (cta == 0 && a.trace_cap > 0) {
                    double* t = a.trace + (size_t)((sc.iter_total - 1) % a.trace_cap) * kTraceWidth;
                    t[0] = r_res; t[1] = s_res; t[2] = sc.beta; t[3] = sc.alpha; t[4] = (double)event;
                }
                s_ratio = ratio;
                s_ctl = ctl;
                if (event & 3) publish_params();  // beta or alpha changed (FP64 log and quotient)
            }
        } else {
            // meanwhile the other warps load the next gather weights w = u'
            // + d (w_s is not read again before phase A); WIDE: and clear
            // this CTA's histogram, which every CTA has read in phase B
            #pragma unroll 16
            for (int e = tid - 32; e < E; e += kIterThreads - 32) {
                w_s[e] = __ldcg(&a.w_next[e]);
                if (WIDE) __stcg(&h64[e], 0ull);
            }
        }
        __syncthreads();
        // commit the slice's new prices (scaled with beta); when beta changed,
        // rescale the gather weights' price part: w = ratio u' + d = w +
        // (ratio - 1) u' (the rescale keeps d, a primal quantity)
        const float ratio = s_ratio;
        const int ctl = s_ctl;
        for (int e = e_lo + tid; e < e_hi; e += kIterThreads) s_u[e - e_lo] = s_un[e - e_lo] * ratio;
        if (ratio != 1.f) {
            #pragma unroll 4
            for (int e = tid; e < E; e += kIterThreads) w_s[e] = fmaf(__ldcg(&a.u_next[e]), ratio - 1.f, w_s[e]);
        }
        __syncthreads();
        if (ctl != 0) break;  // numeric failure (status set) or the stop rule fired
    }
    __syncthreads();
    for (int e = e_lo + tid; e < e_hi; e += kIterThreads) a.u[e] = s_u[e - e_lo];
    if (cta == 0) {
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

template <int G, bool DET, int KL = kMaxPathsPerLane>
cudaError_t launch_iter_t(const IterArgs& a, int grid, cudaStream_t st) {
    const size_t smem = iter_smem_bytes(a.L.E, grid, DET);
    cudaError_t err = cudaFuncSetAttribute(k_iter<G, DET, false, false, uint16_t, KL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    IterArgs args = a;
    const IterArgs* none = nullptr;
    int group = 0;
    void* params[] = {&args, &none, &group};
    return cudaLaunchCooperativeKernel((const void*)k_iter<G, DET, false, false, uint16_t, KL>, dim3(grid),
                                       dim3(kIterThreads), params, smem, st);
}

template <int G, typename IdT, int KL = kMaxPathsPerLane>
cudaError_t launch_iter_wide_t(const IterArgs& a, int grid, cudaStream_t st) {
    const size_t smem = iter_smem_bytes_wide(a.L.E, grid, (int)sizeof(IdT));
    cudaError_t err = cudaFuncSetAttribute(k_iter<G, true, false, true, IdT, KL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    IterArgs args = a;
    const IterArgs* none = nullptr;
    int group = 0;
    void* params[] = {&args, &none, &group};
    return cudaLaunchCooperativeKernel((const void*)k_iter<G, true, false, true, IdT, KL>, dim3(grid),
                                       dim3(kIterThreads), params, smem, st);
}

template <int G, typename IdT>
cudaError_t occupancy_wide_t(int E, int grid_hint, int* blocks) {
    const size_t smem = iter_smem_bytes_wide(E, grid_hint, (int)sizeof(IdT));
    cudaError_t err = cudaFuncSetAttribute(k_iter<G, true, false, true, IdT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_iter<G, true, false, true, IdT>, kIterThreads,
                                                         smem);
}

template <int G>
cudaError_t launch_iter_grouped_t(const IterArgs* args_dev, int n, int group, int E, cudaStream_t st) {
    const size_t smem = iter_smem_bytes(E, group, true);
    cudaError_t err =
        cudaFuncSetAttribute(k_iter<G, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    IterArgs unused{};
    void* params[] = {&unused, &args_dev, &group};
    return cudaLaunchCooperativeKernel((const void*)k_iter<G, true, true>, dim3(n * group), dim3(kIterThreads),
                                       params, smem, st);
}

template <int G, bool DET>
cudaError_t occupancy_t(int E, int grid_hint, int* blocks) {
    const size_t smem = iter_smem_bytes(E, grid_hint, DET);
    cudaError_t err =
        cudaFuncSetAttribute(k_iter<G, DET, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_iter<G, DET, false>, kIterThreads, smem);
}

}  // namespace

// Dynamic shared memory of the iteration kernel: histogram (8 B per edge
// deterministic, 4 B otherwise), gather weights (4 B per edge), staging
// buffers, and the CTA's price slice (current and next) for a grid of at
// least `grid` CTAs.
size_t iter_smem_bytes(int E, int grid, bool det) {
    size_t b = (det ? 2 : 1) * (size_t)(E + 1) * sizeof(unsigned) + (size_t)(E + 1) * sizeof(float);
    b = (b + 31 * sizeof(float) + 127) & ~size_t(127);
    b += (size_t)kIterWarps * 2 * kIterStageRows * kLanes * sizeof(uint16_t);
    const int slice = (E + grid - 1) / (grid > 0 ? grid : 1) + 1;
    b += 2 * (size_t)slice * sizeof(float);
    return b;
}

size_t iter_smem_bytes_wide(int E, int grid, int id_bytes) {
    size_t b = (size_t)kIterWarps * 2 * kIterStageRows * kLanes * (size_t)id_bytes;
    const int slice = (E + grid - 1) / (grid > 0 ? grid : 1) + 1;
    b += 2 * (size_t)slice * sizeof(float);
    return b;
}

cudaError_t iter_occupancy_wide(int G, int id_bytes, int E, int grid_hint, int* blocks_per_sm) {
    if (id_bytes == 4) {
        switch (G) {
            case 1: return occupancy_wide_t<1, uint32_t>(E, grid_hint, blocks_per_sm);
            case 2: return occupancy_wide_t<2, uint32_t>(E, grid_hint, blocks_per_sm);
            case 4: return occupancy_wide_t<4, uint32_t>(E, grid_hint, blocks_per_sm);
            default: return occupancy_wide_t<8, uint32_t>(E, grid_hint, blocks_per_sm);
        }
    }
    switch (G) {
        case 1: return occupancy_wide_t<1, uint16_t>(E, grid_hint, blocks_per_sm);
        case 2: return occupancy_wide_t<2, uint16_t>(E, grid_hint, blocks_per_sm);
        case 4: return occupancy_wide_t<4, uint16_t>(E, grid_hint, blocks_per_sm);
        default: return occupancy_wide_t<8, uint16_t>(E, grid_hint, blocks_per_sm);
    }
}

cudaError_t iter_occupancy(int G, bool det, int E, int grid_hint, int* blocks_per_sm) {
    if (det) {
        switch (G) {
            case 1: return occupancy_t<1, true>(E, grid_hint, blocks_per_sm);
            case 2: return occupancy_t<2, true>(E, grid_hint, blocks_per_sm);
            case 4: return occupancy_t<4, true>(E, grid_hint, blocks_per_sm);
            default: return occupancy_t<8, true>(E, grid_hint, blocks_per_sm);
        }
    }
    switch (G) {
        case 1: return occupancy_t<1, false>(E, grid_hint, blocks_per_sm);
        case 2: return occupancy_t<2, false>(E, grid_hint, blocks_per_sm);
        case 4: return occupancy_t<4, false>(E, grid_hint, blocks_per_sm);
        default: return occupancy_t<8, false>(E, grid_hint, blocks_per_sm);
    }
}

cudaError_t launch_iter(const IterArgs& a, int grid, cudaStream_t st) {
    if (a.hist64 && a.L.id_bytes == 4) {
        switch (a.L.G) {
            case 1:
                return a.L.kl == 1 ? launch_iter_wide_t<1, uint32_t, 1>(a, grid, st)
                                   : launch_iter_wide_t<1, uint32_t>(a, grid, st);
            case 2: return launch_iter_wide_t<2, uint32_t>(a, grid, st);
            case 4: return launch_iter_wide_t<4, uint32_t>(a, grid, st);
            default: return launch_iter_wide_t<8, uint32_t>(a, grid, st);
        }
    }
    if (a.hist64) {
        switch (a.L.G) {
            case 1:
                return a.L.kl == 1 ? launch_iter_wide_t<1, uint16_t, 1>(a, grid, st)
                                   : launch_iter_wide_t<1, uint16_t>(a, grid, st);
            case 2: return launch_iter_wide_t<2, uint16_t>(a, grid, st);
            case 4: return launch_iter_wide_t<4, uint16_t>(a, grid, st);
            default: return launch_iter_wide_t<8, uint16_t>(a, grid, st);
        }
    }
    if (a.L.id_bytes != 2) return cudaErrorInvalidValue;
    if (a.o.deterministic) {
        switch (a.L.G) {
            case 1:
                // one path per lane (single-path demands): the one-slot block code
                return a.L.kl == 1 ? launch_iter_t<1, true, 1>(a, grid, st) : launch_iter_t<1, true>(a, grid, st);
            case 2: return launch_iter_t<2, true>(a, grid, st);
            case 4: return launch_iter_t<4, true>(a, grid, st);
            default: return launch_iter_t<8, true>(a, grid, st);
        }
    }
    switch (a.L.G) {
        case 1: return launch_iter_t<1, false>(a, grid, st);
        case 2: return launch_iter_t<2, false>(a, grid, st);
        case 4: return launch_iter_t<4, false>(a, grid, st);
        default: return launch_iter_t<8, false>(a, grid, st);
    }
}

cudaError_t launch_iter_grouped(const IterArgs* args_dev, int n, int group, int G, int E, cudaStream_t st) {
    switch (G) {
        case 1: return launch_iter_grouped_t<1>(args_dev, n, group, E, st);
        case 2: return launch_iter_grouped_t<2>(args_dev, n, group, E, st);
        case 4: return launch_iter_grouped_t<4>(args_dev, n, group, E, st);
        default: return launch_iter_grouped_t<8>(args_dev, n, group, E, st);
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

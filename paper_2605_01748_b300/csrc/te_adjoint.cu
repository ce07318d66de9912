// Reverse-mode step of the iteration for te_gradient (the differentiated
// form, not in the paper): the adjoint of one fixed-schedule iteration
// (beta and alpha fixed) on the sliced layout.  Forward states are FP32 (the
// iteration kernel's); adjoints are FP64.
//
// One iteration maps (x, u, d) to (x', u', d'), with w = u + d:
//   m_r  = x_r - (1/n_r) sum_{e in r} w_e
//   x'_r = max(0, m_r + nu / n_r), nu the demand's scaled multiplier
//   L_e  = sum_{r ni e} x'_r,  u'_e = max(0, u_e + (L_e - C_e)/n_e),  d' = u' - u
// and its adjoint, from (xb', ub', db') to (xb, ub, db) and the capacity and
// demand adjoints:
//   ub'' = ub' + db';  ub = -db' + [u'_e > 0] ub'';  Lb_e = [u'_e > 0] ub''/n_e;
//   Cb_e -= [u'_e > 0] ub''/n_e
//   gb_r = xb'_r + sum_{e in r} Lb_e
//   on the active set A (x'_r > 0) of a demand, with a_r = 1/n_r, H = sum_A a,
//   S = sum_A x', G = sum_A gb a: if the demand cap binds (S = D_c)
//   dnu/dm_s = -1/H and Db += G/H, else (beta nu = U'(S))
//   (whether the cap binds is the forward step's own decision, read back from
//   its multiplier: binding iff beta nu <= U'(D_c))
//   dnu/dm_s = -alpha nu / (S + alpha nu H); mb_s = gb_s + G dnu/dm_s on A, 0 off A
//   xb = mb;  ub_e += sum_{r ni e} (-mb_r/n_r);  db_e = the same sum
// The last sums (the adjoint of w) are exact 64-bit fixed-point integer sums
// of the terms -mb_r/n_r, each rounded to the nearest multiple of 2^-k where
// 2^k is the largest power of two that keeps every edge's sum below 2^61
// given the step's largest term: order-free, so te_gradient is
// deterministic.  The objective J is summed in a fixed order.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "te_adjoint.h"

namespace te {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < 1 ? 1 : b);
}

// per-edge part before the per-demand step
__global__ void k_adj_edges_in(int E, double* ub, double* db, const float* u1, const float* ne_f,
                               const float* inv_ne, double* Lb, double* Cb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double tot = ub[e] + db[e];
    double uin = -db[e];
    double lb = 0.0;
    if (ne_f[e] > 0.f && u1[e] > 0.f) {
        uin += tot;
        lb = tot * (double)inv_ne[e];
        Cb[e] -= lb;
    }
    Lb[e] = lb;
    ub[e] = uin;
    db[e] = 0.0;
}

// per-demand step: one thread per demand slot.  xb (per path lane) is read
// as the adjoint of x' and overwritten with the adjoint of x; qb receives
// each path's term of the adjoint of w (-mb/n, 0 off the active set) and
// qmax the largest |qb| (zeroed by the caller).
template <typename IdT>
__global__ void k_adj_demands(Layout L, const float* __restrict__ x1, const float* __restrict__ lam1,
                              const double* __restrict__ Lb, double* xb, double* qb, unsigned long long* qmax,
                              double* Db, float beta, float alpha) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * L.dpb) return;
    const int np = L.np[i];
    if (np == 0) return;
    const int b = (int)(i / L.dpb), t = (int)(i % L.dpb);
    const int s0 = L.slotbase[b];
    const IdT* ids = static_cast<const IdT*>(L.ids);
    // pass 1: active set sums
    double S = 0.0, H = 0.0, G = 0.0;
    int na = 0;
    for (int p = 0; p < np; ++p) {
        const size_t sl = (size_t)(s0 + p / L.G);
        const int lane = t * L.G + p % L.G;
        const size_t at = sl * kLanes + lane;
        const float xn = x1[at];
        if (!(xn > 0.f)) continue;
        double g = xb[at];
        int n = 0;
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const int id = ids[(size_t)r * kLanes + lane];
            if (id == L.E) continue;
            g += Lb[id];
            ++n;
        }
        const double a = 1.0 / (double)n;
        S += (double)xn;
        H += a;
        G += g * a;
        ++na;
    }
    // Whether the cap binds is the forward step's decision: it took the cap
    // branch iff its multiplier lambda = beta nu is at most U'(D), where the
    // target (beta nu)^(-1/alpha) reaches D (alpha = 0: lambda = 1 on the
    // slack branch).  lambda is the FP32 value the step stored, so only a
    // demand within a few units in the last place of the kink can be read
    // on the other side.  On the slack branch the multiplier used is
    // U'(S) / beta, which avoids taking nu from x' - m (that difference
    // cancels when the consensus target m is large).
    double dnu = 0.0;  // d nu / d m_s on the active set
    if (na > 0) {
        const double D = (double)L.Dn[i];
        const double lam = (double)lam1[i];
        const bool binds = alpha == 0.f ? lam < 1.0 - 1e-6 : lam * exp((double)alpha * log(D)) <= 1.0;
        if (binds) {
            dnu = -1.0 / H;
            Db[i] += G / H;
        } else {
            const double nu = (alpha == 0.f ? 1.0 : exp(-(double)alpha * log(S))) / (double)beta;
            dnu = -(double)alpha * nu / (S + (double)alpha * nu * H);
        }
    }
    // pass 2: adjoints of x and w
    for (int p = 0; p < np; ++p) {
        const size_t sl = (size_t)(s0 + p / L.G);
        const int lane = t * L.G + p % L.G;
        const size_t at = sl * kLanes + lane;
        double mb = 0.0;
        int n = 0;
        if (x1[at] > 0.f) {
            double g = xb[at];
            for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                const int id = ids[(size_t)r * kLanes + lane];
                if (id == L.E) continue;
                g += Lb[id];
                ++n;
            }
            mb = g + G * dnu;
        }
        xb[at] = mb;
        const double q = mb != 0.0 ? -mb / (double)n : 0.0;
        qb[at] = q;
        // |q| as the bits of a non-negative double: their order is the
        // numbers' order, so the maximum does not depend on the order either
        if (q != 0.0) atomicMax(qmax, (unsigned long long)__double_as_longlong(fabs(q)));
    }
}

// The fixed-point scale 2^k of a step: the largest k with 2^k max|qb| <
// 2^(61 - deg_bits), so that each term is below 2^(61 - deg_bits) and each
// edge's sum of at most 2^deg_bits terms below 2^61 in magnitude.  0 when
// every term is 0; NaN when a term is not finite (the gradient then is NaN).
__device__ __forceinline__ double adj_scale(unsigned long long qmax_bits, int deg_bits) {
    const double m = __longlong_as_double((long long)qmax_bits);
    if (!(m < INFINITY)) return NAN;
    if (!(m > 0.0)) return 0.0;
    int e = 0;
    frexp(m, &e);  // m < 2^e
    return ldexp(1.0, min(61 - deg_bits - e, 1000));
}

// the adjoint of w per edge: one thread per path lane adds its paths' terms
// as fixed-point integers
template <typename IdT>
__global__ void k_adj_scatter(Layout L, const double* __restrict__ qb, const unsigned long long* qmax, int deg_bits,
                              unsigned long long* wfix) {
    const double scale = adj_scale(*qmax, deg_bits);
    if (!(scale > 0.0)) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * kLanes) return;
    const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    const IdT* ids = static_cast<const IdT*>(L.ids);
    for (int j = 0; j < KB; ++j) {
        const size_t sl = (size_t)(s0 + j);
        const double v = qb[sl * kLanes + lane];
        if (v == 0.0) continue;
        const unsigned long long q = (unsigned long long)llrint(v * scale);  // two's complement
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const int id = ids[(size_t)r * kLanes + lane];
            if (id != L.E) atomicAdd(&wfix[id], q);
        }
    }
}

// per-edge part after the per-demand step: w = u + d
__global__ void k_adj_edges_out(int E, double* ub, double* db, unsigned long long* wfix,
                                const unsigned long long* qmax, int deg_bits) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double scale = adj_scale(*qmax, deg_bits);
    const double wb = scale > 0.0 ? (double)(long long)wfix[e] / scale : (scale == 0.0 ? 0.0 : scale);
    ub[e] += wb;
    db[e] = wb;
    wfix[e] = 0ull;
}

// objective terms U_alpha(scale S_c) of the iterate x into Uc, and the
// adjoint dJ/dx_r = scale U'(scale S_c) on every path of demand c
__global__ void k_adj_objective(Layout L, const float* __restrict__ x, double alpha, double scale, double* xb,
                                double* Uc) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * L.dpb) return;
    const int np = L.np[i];
    if (np == 0) return;
    const int b = (int)(i / L.dpb), t = (int)(i % L.dpb);
    const int s0 = L.slotbase[b];
    double S = 0.0;
    for (int p = 0; p < np; ++p) S += (double)x[(size_t)(s0 + p / L.G) * kLanes + t * L.G + p % L.G];
    const double v = scale * S;
    const double U = alpha == 1.0 ? log(v) : (pow(v, 1.0 - alpha) - 1.0) / (1.0 - alpha);
    const double g = scale * (alpha == 0.0 ? 1.0 : exp(-alpha * log(v)));
    for (int p = 0; p < np; ++p) xb[(size_t)(s0 + p / L.G) * kLanes + t * L.G + p % L.G] = g;
    Uc[i] = U;
}

// acc[0] = sum of v[0..n) in a fixed order (one CTA: strided sums per
// thread, then the threads' sums in thread order)
__global__ void k_sum_ordered(const double* v, long long n, double* acc) {
    __shared__ double part[kThreads];
    double a = 0.0;
    for (long long i = threadIdx.x; i < n; i += kThreads) a += v[i];
    part[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads; ++k) t += part[k];
        acc[0] = t;
    }
}

// initial state x^0_r = D_c / |P_c|: its adjoint into the demand's
__global__ void k_adj_initial(Layout L, const double* xb, double* Db) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * L.dpb) return;
    const int np = L.np[i];
    if (np == 0) return;
    const int b = (int)(i / L.dpb), t = (int)(i % L.dpb);
    const int s0 = L.slotbase[b];
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += xb[(size_t)(s0 + p / L.G) * kLanes + t * L.G + p % L.G];
    Db[i] += s / (double)np;
}

// gradients in caller order and units
__global__ void k_adj_out(Layout L, const double* Cb, const double* Db, double inv_scale, double* gC, double* gD) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < L.E) gC[i] = Cb[i] * inv_scale;
    if (i < (long long)L.nblocks * L.dpb) {
        const int c = L.demand_of[i];
        if (c >= 0) gD[c] = Db[i] * inv_scale;
    }
}

}  // namespace

cudaError_t adjoint_step(const Layout& L, const float* xk, const float* x1, const float* uk1, const float* wk,
                         const float* lam1, float beta, float alpha, AdjointBuffers& B, cudaStream_t st) {
    k_adj_edges_in<<<grid_for(L.E), kThreads, 0, st>>>(L.E, B.ub, B.db, uk1, L.ne_f, L.inv_ne, B.Lb, B.Cb);
    (void)xk;
    (void)wk;
    cudaError_t err = cudaMemsetAsync(B.qmax, 0, sizeof(unsigned long long), st);
    if (err != cudaSuccess) return err;
    const unsigned gd = grid_for((long long)L.nblocks * L.dpb), gs = grid_for((long long)L.nblocks * kLanes);
    if (L.id_bytes == 4) {  // more than 65,534 edges
        k_adj_demands<uint32_t><<<gd, kThreads, 0, st>>>(L, x1, lam1, B.Lb, B.xb, B.qb, B.qmax, B.Db, beta, alpha);
        k_adj_scatter<uint32_t><<<gs, kThreads, 0, st>>>(L, B.qb, B.qmax, B.deg_bits, B.wfix);
    } else {
        k_adj_demands<uint16_t><<<gd, kThreads, 0, st>>>(L, x1, lam1, B.Lb, B.xb, B.qb, B.qmax, B.Db, beta, alpha);
        k_adj_scatter<uint16_t><<<gs, kThreads, 0, st>>>(L, B.qb, B.qmax, B.deg_bits, B.wfix);
    }
    k_adj_edges_out<<<grid_for(L.E), kThreads, 0, st>>>(L.E, B.ub, B.db, B.wfix, B.qmax, B.deg_bits);
    return cudaGetLastError();
}

cudaError_t adjoint_objective(const Layout& L, const float* x, double alpha, double scale, AdjointBuffers& B,
                              cudaStream_t st) {
    const long long nd = (long long)L.nblocks * L.dpb;
    k_adj_objective<<<grid_for(nd), kThreads, 0, st>>>(L, x, alpha, scale, B.xb, B.Uc);
    k_sum_ordered<<<1, kThreads, 0, st>>>(B.Uc, nd, B.acc);
    return cudaGetLastError();
}

cudaError_t adjoint_finish(const Layout& L, double scale, AdjointBuffers& B, double* gC, double* gD,
                           cudaStream_t st) {
    k_adj_initial<<<grid_for((long long)L.nblocks * L.dpb), kThreads, 0, st>>>(L, B.xb, B.Db);
    const long long n = std::max<long long>((long long)L.E, (long long)L.nblocks * L.dpb);
    k_adj_out<<<grid_for(n), kThreads, 0, st>>>(L, B.Cb, B.Db, 1.0 / scale, gC, gD);
    return cudaGetLastError();
}

}  // namespace te

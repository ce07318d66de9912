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
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "te_internal.cuh"

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
// as the adjoint of x' and overwritten with the adjoint of x; wbar collects
// the adjoint of w (zeroed by the caller).
__global__ void k_adj_demands(Layout L, const float* __restrict__ x1, const float* __restrict__ lam1,
                              const double* __restrict__ Lb, double* xb, double* wbar, double* Db, float beta,
                              float alpha) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * L.dpb) return;
    const int np = L.np[i];
    if (np == 0) return;
    const int b = (int)(i / L.dpb), t = (int)(i % L.dpb);
    const int s0 = L.slotbase[b];
    const uint16_t* ids = static_cast<const uint16_t*>(L.ids);
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
        if (mb != 0.0) {
            const double qb = -mb / (double)n;
            for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                const int id = ids[(size_t)r * kLanes + lane];
                if (id != L.E) atomicAdd(&wbar[id], qb);
            }
        }
    }
}

// per-edge part after the per-demand step: w = u + d
__global__ void k_adj_edges_out(int E, double* ub, double* db, double* wbar) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    ub[e] += wbar[e];
    db[e] = wbar[e];
    wbar[e] = 0.0;
}

// objective J = sum_c U_alpha(scale S_c) of the iterate x, and the adjoint
// dJ/dx_r = scale U'(scale S_c) on every path of demand c; J accumulates
// into acc[0]
__global__ void k_adj_objective(Layout L, const float* __restrict__ x, double alpha, double scale, double* xb,
                                double* acc) {
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
    atomicAdd(acc, U);
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
    k_adj_demands<<<grid_for((long long)L.nblocks * L.dpb), kThreads, 0, st>>>(L, x1, lam1, B.Lb, B.xb, B.wbar, B.Db,
                                                                             beta, alpha);
    k_adj_edges_out<<<grid_for(L.E), kThreads, 0, st>>>(L.E, B.ub, B.db, B.wbar);
    return cudaGetLastError();
}

cudaError_t adjoint_objective(const Layout& L, const float* x, double alpha, double scale, AdjointBuffers& B,
                              cudaStream_t st) {
    k_adj_objective<<<grid_for((long long)L.nblocks * L.dpb), kThreads, 0, st>>>(L, x, alpha, scale, B.xb, B.acc);
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

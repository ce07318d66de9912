// Feasibility projection of GATE (Algorithm 2, Section 3.5) on the sliced
// device layout, plus the gathers between the sliced layout and the caller's
// path order.
//
// Steps (all on a copy of the iterate, normalised units):
//   1. x <- max(x, 0); S_c, L_e, V_e = max(L_e - C_e, 0), C_p = number of
//      violated edges on p.
//   2. Demand step: every demand with S_c > D_c trims its paths greedily in
//      descending score S_c^alpha * C_p.  Inside one demand S_c is common, so
//      the order is descending C_p, ties to the lower path index.
//   3. Recompute S_c, L_e, V_e, C_p.
//   4. Capacity step: every violated edge plans, from this one snapshot, the
//      trims of its paths in descending score (ties to the lower path index)
//      until V_e is covered; each path then loses the largest trim planned
//      for it over its edges.  Each edge's load drops by at least V_e, so the
//      result is feasible.  The plan of an edge is found without sorting: a
//      radix select over the 64-bit key (score bits, then inverted path
//      index) finds the threshold path at which the running sum of rates in
//      key order reaches V_e; paths above it are trimmed in full and the
//      threshold path by the remainder.  The select passes read a list of
//      the violated incidences (one entry per violated edge of a path with
//      a rate), formed once, instead of walking every path's edge ids.
// Scores are compared as keys: alpha*log(S_c) + log(C_p) evaluated in FP64
// with S_c in the caller's units and rounded to FP32 (the oracle forms the
// same key, so both order the paths alike up to FP64 rounding at an FP32
// boundary).
//
// Edge loads and the radix-select histograms are sums over many paths; they
// are accumulated as 64-bit integers in units of 2^-40 (normalised
// rates), so the sums do not depend on the order of the atomics and two
// projections of the same iterate return the same bits.  Rounding is
// conservative: a rate enters the loads rounded up (a violation is never
// missed, never under-estimated) and the histograms rounded down (the trims
// cover at least the violation).
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "te_internal.cuh"
#include "te_proj.h"

namespace te {
namespace {

constexpr int kThreads = 256;
// 2^-40 resolution; a load of up to 2^23 normalised units fits in 63 bits
// (te_create bounds the demand through an edge far below that)
constexpr double kFixScale = 1099511627776.0;  // 2^40

__device__ __forceinline__ unsigned long long fix_up(float v) {
    return (unsigned long long)ceil((double)v * kFixScale);
}
__device__ __forceinline__ unsigned long long fix_down(float v) {
    return (unsigned long long)floor((double)v * kFixScale);
}
// integer sum back to normalised units, rounded up / down
__device__ __forceinline__ double unfix_up(unsigned long long q) { return __ull2double_ru(q) * (1.0 / kFixScale); }
__device__ __forceinline__ double unfix_down(unsigned long long q) { return __ull2double_rd(q) * (1.0 / kFixScale); }

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 1048576) b = 1048576;
    return (unsigned)b;
}

template <typename IdT>
__device__ __forceinline__ const IdT* ids_of(const Layout& L) {
    return static_cast<const IdT*>(L.ids);
}

// x <- max(x, 0) on every slot; S = the demand's total, written to each of
// its G lanes.  One thread per demand.
__global__ void k_clamp_sum(Layout L, float* x, double* S) {
    const int DPB = L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * DPB) return;
    const int b = (int)(i / DPB), t = (int)(i % DPB);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    double acc = 0.0;
    for (int hh = 0; hh < L.G; ++hh) {
        const int lane = t * L.G + hh;
        for (int j = 0; j < KB; ++j) {
            float* p = &x[(size_t)(s0 + j) * kLanes + lane];
            const float v = fmaxf(*p, 0.f);
            *p = v;
            acc += (double)v;
        }
    }
    S[i] = acc;
}

// L_e = sum of rates over the paths through e, each rounded up to the
// fixed-point unit (loads must be zeroed).
template <typename IdT>
__global__ void k_loads(Layout L, const float* x, unsigned long long* loads) {
    const IdT* ids = ids_of<IdT>(L);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * kLanes) return;
    const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    for (int j = 0; j < KB; ++j) {
        const size_t sl = (size_t)(s0 + j);
        const float v = x[sl * kLanes + lane];
        if (v == 0.f) continue;
        const unsigned long long q = fix_up(v);
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const IdT id = ids[(size_t)r * kLanes + lane];
            if ((int)id != L.E) atomicAdd(&loads[id], q);
        }
    }
}

// V_e > 0 flags, compact indices of violated edges and their violation.
// The compact index of an edge depends on the order of the atomics, but every
// result below is computed per edge and does not depend on it.
__global__ void k_viol(Layout L, const unsigned long long* loads, unsigned char* viol, int* vidx, int* nviol,
                       double* rem, unsigned long long* prefix) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.E) return;
    const double V = unfix_up(loads[e]) - (double)L.cap_n[e];
    if (V > 0.0) {
        viol[e] = 1;
        const int v = atomicAdd(nviol, 1);
        vidx[e] = v;
        rem[v] = V;
        prefix[v] = 0ull;
    } else {
        viol[e] = 0;
        vidx[e] = -1;
    }
}

// C_p = number of violated edges on each path.
template <typename IdT>
__global__ void k_count_viol(Layout L, const unsigned char* viol, unsigned char* Cp) {
    const IdT* ids = ids_of<IdT>(L);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * kLanes) return;
    const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    for (int j = 0; j < KB; ++j) {
        const size_t sl = (size_t)(s0 + j);
        int c = 0;
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const IdT id = ids[(size_t)r * kLanes + lane];
            if ((int)id != L.E) c += viol[id];
        }
        Cp[sl * kLanes + lane] = (unsigned char)(c > 255 ? 255 : c);
    }
}

// Demand step: trims S_c - D_c from the demand's paths in descending C_p,
// ties to the lower path index.  One thread per demand; path p of the demand
// is on lane t*G + p%G, slot p/G.
__global__ void k_demand_trim(Layout L, float* x, const double* S, const unsigned char* Cp) {
    const int DPB = L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * DPB) return;
    const int b = (int)(i / DPB), t = (int)(i % DPB);
    const double D = (double)L.Dn[i];
    double Ec = S[i] - D;
    if (!(Ec > 0.0) || D <= 0.0) return;
    const int s0 = L.slotbase[b];
    const int np = L.np[i];
    // paths without a rate lose nothing; leaving them out does not change
    // the order of the others
    unsigned taken = 0u;  // np <= 32
    for (int p = 0; p < np; ++p)
        if (x[(size_t)(s0 + p / L.G) * kLanes + t * L.G + p % L.G] == 0.f) taken |= 1u << p;
    for (int k = 0; k < np && Ec > 0.0; ++k) {
        int best = -1, bc = -1;
        for (int p = 0; p < np; ++p) {
            if (taken & (1u << p)) continue;
            const int c = Cp[(size_t)(s0 + p / L.G) * kLanes + t * L.G + p % L.G];
            if (c > bc) { bc = c; best = p; }
        }
        if (best < 0) break;
        taken |= 1u << best;
        float* q = &x[(size_t)(s0 + best / L.G) * kLanes + t * L.G + best % L.G];
        const double d = fmin(Ec, (double)*q);
        *q = d >= (double)*q ? 0.f : __double2float_rd((double)*q - d);
        Ec -= d;
    }
}

__device__ __forceinline__ unsigned orderable(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The two terms of the paths' scores, formed once per projection (FP64
// logarithms are slow on this part, and the select passes read the keys nine
// times): score[c] = alpha log(S_c scale) for every demand c (0 for alpha =
// 0, -inf for S_c = 0), and score[nd + k] = log(k) for k = 0..255 (C_p is a
// byte).  One thread per demand; the first 256 threads also fill the table.
__global__ void k_score_terms(Layout L, const double* S, double alpha, double scale, double* score) {
    const long long nd = (long long)L.nblocks * L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < 256) score[nd + i] = log((double)i);
    if (i >= nd) return;
    score[i] = alpha == 0.0 ? 0.0 : (S[i] > 0.0 ? alpha * log(S[i] * scale) : -INFINITY);
}

// Key of a path: high word = orderable(FP32 of alpha log S_c + log C_p), S_c
// in caller units (S normalised times scale), low word = inverted caller
// path index (lower index ranks first among equal scores).  aS is the
// demand's score term and logc the table of k_score_terms.
__device__ __forceinline__ unsigned long long path_key(double aS, int Cp, const double* logc, long long user_path) {
    const float ls = (Cp <= 0 || aS == -INFINITY) ? -INFINITY : (float)(aS + logc[Cp]);
    return ((unsigned long long)orderable(ls) << 32) | (unsigned long long)(0xffffffffu - (unsigned)user_path);
}

// The second round's count of violated edges per path fused with the list
// of violated incidences (see below): each thread counts its paths' violated
// edges, the CTA takes its ranges with one atomic each, and the thread walks
// the rows of its counted paths again (just read) to write their entries and
// path records, but only as far as cap: cursor[0] and cursor[1] end as the
// totals, and when cursor[0] exceeds cap the caller grows the list and
// fills it with k_vlist_fill.
template <typename IdT>
__global__ void k_count_fill(Layout L, const float* x, const unsigned char* viol, const int* vidx,
                             const double* score, unsigned char* Cp, uint4* vlist, uint4* plist,
                             unsigned long long cap, unsigned long long* cursor) {
    constexpr int KL = kMaxPathsPerLane;
    __shared__ unsigned s_warp[kThreads / 32], s_pwarp[kThreads / 32];
    __shared__ unsigned long long s_base, s_pbase;
    const IdT* ids = ids_of<IdT>(L);
    const double* logc = score + (size_t)L.nblocks * L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool valid = i < (long long)L.nblocks * kLanes;
    const int b = valid ? (int)(i / kLanes) : 0, lane = (int)(i % kLanes);
    const int s0 = valid ? L.slotbase[b] : 0, KB = valid ? L.slotbase[b + 1] - s0 : 0;
    int cnt[KL];
    unsigned c = 0u, pc = 0u;  // this thread's entries and paths
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        cnt[j] = 0;
        if (j < KB) {
            const size_t sl = (size_t)(s0 + j);
            int n = 0;
            for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                const IdT id = ids[(size_t)r * kLanes + lane];
                if ((int)id != L.E) n += viol[id];
            }
            n = n > 255 ? 255 : n;
            Cp[sl * kLanes + lane] = (unsigned char)n;
            if (n != 0 && x[sl * kLanes + lane] != 0.f) {
                cnt[j] = n;
                c += (unsigned)n;
                ++pc;
            }
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned incl = c, pincl = pc;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        const unsigned py = __shfl_up_sync(0xffffffffu, pincl, o);
        if (l >= o) {
            incl += y;
            pincl += py;
        }
    }
    if (l == 31) {
        s_warp[w] = incl;
        s_pwarp[w] = pincl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull, pt = 0ull;
        for (int k = 0; k < kThreads / 32; ++k) {
            const unsigned v = s_warp[k], pv = s_pwarp[k];
            s_warp[k] = (unsigned)t;
            s_pwarp[k] = (unsigned)pt;
            t += v;
            pt += pv;
        }
        s_base = t != 0ull ? atomicAdd(&cursor[0], t) : 0ull;
        s_pbase = pt != 0ull ? atomicAdd(&cursor[1], pt) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = s_base + s_warp[w] + (incl - c);
    unsigned long long ppos = s_pbase + s_pwarp[w] + (pincl - pc);
    if (pos + c > cap) return;  // the list is too short: the caller fills it again
    #pragma unroll
    for (int j = 0; j < KL; ++j) {
        if (cnt[j] == 0) continue;
        const size_t sl = (size_t)(s0 + j);
        const float v = x[sl * kLanes + lane];
        const unsigned long long key = path_key(score[(size_t)b * L.dpb + lane / L.G], cnt[j], logc,
                                                L.slot_path[sl * kLanes + lane]);
        if (ppos < cap) plist[ppos] = make_uint4((unsigned)pos, (unsigned)cnt[j], (unsigned)(sl * kLanes + lane), 0u);
        ++ppos;
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const IdT id = ids[(size_t)r * kLanes + lane];
            if ((int)id == L.E) continue;
            const int vi = vidx[id];
            if (vi < 0) continue;
            if (pos < cap)
                vlist[pos] = make_uint4((unsigned)key, (unsigned)(key >> 32), __float_as_uint(v), (unsigned)vi);
            ++pos;
        }
    }
}

// The violated incidences of the capacity step: for every path with a rate
// and a violated edge, one entry per violated edge on it, (key low word, key
// high word, rate bits, compact edge index), as many as the sum of C_p over
// the paths with a rate.  k_count_fill and k_vlist_fill write them, each CTA
// into a range taken with one atomic; the order of the entries therefore
// varies between runs, but the histograms they feed are integer sums.
// k_vlist_fill runs on a grid of a few CTAs per SM, each thread taking lanes
// i, i + (grid threads), ..., so that the shared counters see one atomic per
// CTA.
template <typename IdT>
__global__ void k_vlist_fill(Layout L, const float* x, const double* score, const unsigned char* Cp,
                             const int* vidx, uint4* vlist, uint4* plist, unsigned long long cap,
                             unsigned long long* cursor) {
    __shared__ unsigned s_warp[kThreads / 32], s_pwarp[kThreads / 32];
    __shared__ unsigned long long s_base, s_pbase;
    const IdT* ids = ids_of<IdT>(L);
    const double* logc = score + (size_t)L.nblocks * L.dpb;
    const long long n = (long long)L.nblocks * kLanes, step = (long long)gridDim.x * blockDim.x;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned c = 0u, pc = 0u;  // this thread's entries and paths, over all its lanes
    for (long long i = i0; i < n; i += step) {
        const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
        const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
        for (int j = 0; j < KB; ++j) {
            const size_t k = (size_t)(s0 + j) * kLanes + lane;
            if (x[k] != 0.f && Cp[k] != 0) {
                c += Cp[k];
                ++pc;
            }
        }
    }
    // this thread's offsets in the CTA's ranges: exclusive scans over the CTA
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned incl = c, pincl = pc;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        const unsigned py = __shfl_up_sync(0xffffffffu, pincl, o);
        if (l >= o) {
            incl += y;
            pincl += py;
        }
    }
    if (l == 31) {
        s_warp[w] = incl;
        s_pwarp[w] = pincl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull, pt = 0ull;
        for (int k = 0; k < kThreads / 32; ++k) {
            const unsigned v = s_warp[k], pv = s_pwarp[k];
            s_warp[k] = (unsigned)t;
            s_pwarp[k] = (unsigned)pt;
            t += v;
            pt += pv;
        }
        s_base = t != 0ull ? atomicAdd(&cursor[0], t) : 0ull;
        s_pbase = pt != 0ull ? atomicAdd(&cursor[1], pt) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = s_base + s_warp[w] + (incl - c);
    unsigned long long ppos = s_pbase + s_pwarp[w] + (pincl - pc);
    for (long long i = i0; i < n; i += step) {
        const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
        const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
        for (int j = 0; j < KB; ++j) {
            const size_t sl = (size_t)(s0 + j);
            const float v = x[sl * kLanes + lane];
            const int cp = Cp[sl * kLanes + lane];
            if (v == 0.f || cp == 0) continue;
            const unsigned long long key = path_key(score[(size_t)b * L.dpb + lane / L.G], cp, logc,
                                                    L.slot_path[sl * kLanes + lane]);
            if (ppos < cap) plist[ppos] = make_uint4((unsigned)pos, (unsigned)cp, (unsigned)(sl * kLanes + lane), 0u);
            ++ppos;
            for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
                const IdT id = ids[(size_t)r * kLanes + lane];
                if ((int)id == L.E) continue;
                const int vi = vidx[id];
                if (vi < 0) continue;
                if (pos < cap)
                    vlist[pos] = make_uint4((unsigned)key, (unsigned)(key >> 32), __float_as_uint(v), (unsigned)vi);
                ++pos;
            }
        }
    }
}

// One radix-select pass over the violated incidences: per violated edge,
// histogram of the rates of the candidate paths (keys matching the selected
// prefix) by the next 8-bit digit.
__global__ void k_select_hist_list(const uint4* vlist, unsigned long long n, int E, const unsigned char* done,
                                   const unsigned long long* prefix, unsigned long long* hist, int pass) {
    const int shift = 56 - 8 * pass;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 e = vlist[i];
        const int vi = (int)e.w;
        if (vi < 0 || vi >= E || done[vi]) continue;  // (every entry's index is in range by construction)
        const unsigned long long key = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
        if (pass > 0 && ((key ^ prefix[vi]) >> (shift + 8)) != 0ull) continue;
        atomicAdd(&hist[(size_t)vi * 256 + (int)((key >> shift) & 0xffull)], fix_down(__uint_as_float(e.z)));
    }
}

// Per violated edge: choose the digit at which the running sum (from the top
// digit down) reaches the remaining violation.  The sums are integers (rates
// rounded down), compared with the violation rounded up.  One warp per
// violated edge: lane l holds the digits 255 - 8l - k, k = 0..7 (so lane
// order and k follow the scan from the top digit down), the lanes' sums are
// prefix-summed across the warp, and the first digit with a rate whose
// running sum reaches the violation is the pick; the sum of the digits above
// it becomes the part trimmed in full.
__global__ void k_select_pick(const int* nviol, unsigned long long* hist, unsigned long long* prefix, double* rem,
                              unsigned char* done, int pass) {
    const int v = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int l = threadIdx.x & 31;
    if (v >= *nviol || done[v]) return;  // (the whole warp)
    const int shift = 56 - 8 * pass;
    unsigned long long* h = hist + (size_t)v * 256;
    unsigned long long c[8], sum = 0ull;
    #pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k] = h[255 - 8 * l - k];
        sum += c[k];
    }
    #pragma unroll
    for (int k = 0; k < 8; ++k) h[255 - 8 * l - k] = 0ull;  // ready for the next pass
    unsigned long long incl = sum;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += y;
    }
    unsigned long long cum = incl - sum;  // the digits above this lane's
    const double need = rem[v];
    const unsigned long long need_q = (unsigned long long)ceil(need * kFixScale);
    int hit = -1;
    unsigned long long cum_hit = 0ull;
    #pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (hit < 0 && c[k] > 0ull && cum + c[k] >= need_q) {
            hit = k;
            cum_hit = cum;
        }
        cum += c[k];
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit >= 0);
    if (m == 0u) {
        // rounding left the candidates short of V_e: trim all of them in full
        if (l == 0) done[v] = 2;
        return;
    }
    const int src = __ffs(m) - 1;
    const int k0 = __shfl_sync(0xffffffffu, hit, src);
    const unsigned long long cum0 = __shfl_sync(0xffffffffu, cum_hit, src);
    if (l == 0) {
        prefix[v] |= (unsigned long long)(255 - 8 * src - k0) << shift;
        rem[v] = need - unfix_down(cum0);
    }
}

// Apply, over the path list: every path with a violated edge loses the
// largest trim planned for it by its violated edges (a path at or above its
// edge's threshold key in full, the threshold path by the remainder).
__global__ void k_edge_trim_list(const uint4* plist, const unsigned long long* npaths, const uint4* vlist,
                                 unsigned long long cap, int E, float* x, const unsigned long long* prefix,
                                 const double* rem, const unsigned char* done) {
    const unsigned long long n = *npaths < cap ? *npaths : cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 p = plist[i];
        if ((unsigned long long)p.x + p.y > cap) continue;  // (in range by construction)
        const float v = __uint_as_float(vlist[p.x].z);
        double trim = 0.0;
        for (unsigned k = 0; k < p.y; ++k) {
            const uint4 e = vlist[p.x + k];
            const int vi = (int)e.w;
            if (vi < 0 || vi >= E) continue;
            const unsigned long long key = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
            double t;
            if (done[vi] == 2) {
                // all candidates (keys at or above the chosen prefix) in full
                t = key >= prefix[vi] ? (double)v : 0.0;
            } else if (key > prefix[vi]) {
                t = (double)v;
            } else if (key == prefix[vi]) {
                t = fmin((double)v, rem[vi]);
            } else {
                t = 0.0;
            }
            trim = fmax(trim, t);
        }
        // a full trim leaves exactly zero; a partial one rounds down so the
        // edge ends at or below its capacity
        x[p.z] = trim >= (double)v ? 0.f : __double2float_rd((double)v - trim);
    }
}

__global__ void k_to_user(Layout L, const float* x, float* out, float scale) {
    const long long n = L.nslots * kLanes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = L.slot_path[i];
        if (p >= 0) out[p] = x[i] * scale;
    }
}

__global__ void k_from_user(Layout L, const float* in, float* x, float inv_scale) {
    const long long n = L.nslots * kLanes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = L.slot_path[i];
        x[i] = p >= 0 ? in[p] * inv_scale : 0.f;
    }
}

// ---------------- proportional feasibility scaling (not in the paper) ----------------
// te_allocation with project = 2: every over-served demand is scaled to D_c,
// then every path by the smallest min(1, C_e / L_e) over its edges.  The
// factors are rounded toward zero (FP64 quotient, its FP32 conversion, and
// the FP32 product), so the FP32 result never exceeds a bound the exact
// scaling meets.

// x <- x * D_c / S_c on every path of a demand with S_c > D_c.  One thread
// per demand.
__global__ void k_demand_scale(Layout L, float* x, const double* S) {
    const int DPB = L.dpb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * DPB) return;
    const double D = (double)L.Dn[i];
    if (!(S[i] > D)) return;
    const float g = __double2float_rz(__ddiv_rz(D, S[i]));
    const int b = (int)(i / DPB), t = (int)(i % DPB);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    for (int hh = 0; hh < L.G; ++hh)
        for (int j = 0; j < KB; ++j) {
            float* q = &x[(size_t)(s0 + j) * kLanes + t * L.G + hh];
            *q = __fmul_rz(*q, g);
        }
}

// f_e = min(1, C_e / L_e), L_e rounded up.
__global__ void k_edge_factor(Layout L, const unsigned long long* loads, double* f) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.E) return;
    const double C = (double)L.cap_n[e];
    const double Le = unfix_up(loads[e]);
    f[e] = Le > C ? __ddiv_rz(C, Le) : 1.0;
}

// x_p <- x_p * min_{e in p} f_e.  One thread per lane of a block.
template <typename IdT>
__global__ void k_path_scale(Layout L, float* x, const double* f) {
    const IdT* ids = ids_of<IdT>(L);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)L.nblocks * kLanes) return;
    const int b = (int)(i / kLanes), lane = (int)(i % kLanes);
    const int s0 = L.slotbase[b], KB = L.slotbase[b + 1] - s0;
    for (int j = 0; j < KB; ++j) {
        const size_t sl = (size_t)(s0 + j);
        const float v = x[sl * kLanes + lane];
        if (v == 0.f) continue;
        double g = 1.0;
        for (unsigned r = L.rowoff[sl]; r < L.rowoff[sl + 1]; ++r) {
            const IdT id = ids[(size_t)r * kLanes + lane];
            if ((int)id != L.E) g = fmin(g, f[id]);
        }
        if (g < 1.0) x[sl * kLanes + lane] = __fmul_rz(v, __double2float_rz(g));
    }
}

template <typename IdT>
cudaError_t project_scale_t(const Layout& L, float* x, const ProjScratch& s, cudaStream_t st) {
    const unsigned gl = grid_for((long long)L.nblocks * kLanes, kThreads);
    const unsigned ge = grid_for(L.E, kThreads);
    const unsigned gd = grid_for((long long)L.nblocks * L.dpb, kThreads);
    cudaError_t err;
    k_clamp_sum<<<gd, kThreads, 0, st>>>(L, x, s.S);
    k_demand_scale<<<gd, kThreads, 0, st>>>(L, x, s.S);
    if ((err = cudaMemsetAsync(s.loads, 0, sizeof(unsigned long long) * (size_t)L.E, st)) != cudaSuccess) return err;
    k_loads<IdT><<<gl, kThreads, 0, st>>>(L, x, s.loads);
    k_edge_factor<<<ge, kThreads, 0, st>>>(L, s.loads, s.rem);
    k_path_scale<IdT><<<gl, kThreads, 0, st>>>(L, x, s.rem);
    return cudaGetLastError();
}

template <typename IdT>
cudaError_t project_t(const Layout& L, float* x, double alpha, double scale, ProjScratch& s, cudaStream_t st,
                      int* launched_out) {
    const long long lanes = (long long)L.nblocks * kLanes;
    const unsigned gl = grid_for(lanes, kThreads);
    const unsigned ge = grid_for(L.E, kThreads);
    cudaError_t err;
    const unsigned gd = grid_for((long long)L.nblocks * L.dpb, kThreads);
    for (int round = 0; round < 2; ++round) {
        k_clamp_sum<<<gd, kThreads, 0, st>>>(L, x, s.S);
        if ((err = cudaMemsetAsync(s.loads, 0, sizeof(unsigned long long) * (size_t)L.E, st)) != cudaSuccess)
            return err;
        if ((err = cudaMemsetAsync(s.nviol, 0, sizeof(int), st)) != cudaSuccess) return err;
        k_loads<IdT><<<gl, kThreads, 0, st>>>(L, x, s.loads);
        k_viol<<<ge, kThreads, 0, st>>>(L, s.loads, s.viol, s.vidx, s.nviol, s.rem, s.prefix);
        if (round == 0) {
            k_count_viol<IdT><<<gl, kThreads, 0, st>>>(L, s.viol, s.Cp);
            k_demand_trim<<<gd, kThreads, 0, st>>>(L, x, s.S, s.Cp);
        }
    }
    // capacity step: radix select of each violated edge's threshold path
    unsigned char* done = s.viol;  // reuse: per violated-edge flags (E bytes >= nviol), set after the count
    k_score_terms<<<grid_for((long long)L.nblocks * L.dpb > 256 ? (long long)L.nblocks * L.dpb : 256, kThreads),
                    kThreads, 0, st>>>(L, s.S, alpha, scale, s.score);
    // the second round's counts and the violated incidences in one walk;
    // the totals come back to the host (the one synchronisation of the
    // projection), and a list too short is grown and filled again
    if ((err = cudaMemsetAsync(s.vtotal, 0, 3 * sizeof(unsigned long long), st)) != cudaSuccess) return err;
    k_count_fill<IdT><<<gl, kThreads, 0, st>>>(L, x, s.viol, s.vidx, s.score, s.Cp, s.vlist, s.plist, s.vcap,
                                               s.vtotal + 1);
    int launched = kProjectLaunches;
    unsigned long long total = 0ull;
    if ((err = cudaMemcpyAsync(&total, s.vtotal + 1, sizeof total, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
    if (total >= 0xffffffffull) return cudaErrorInvalidValue;  // entry indices are 32-bit
    if (total > s.vcap) {
        if (s.vlist) cudaFree(s.vlist);
        s.vlist = nullptr;
        s.plist = nullptr;
        s.vcap = 0;
        const unsigned long long cap = total + total / 4 + 1024;
        // entries, then as many path records (a path has at least one entry)
        if ((err = cudaMalloc(&s.vlist, 2 * sizeof(uint4) * (size_t)cap)) != cudaSuccess) return err;
        s.plist = s.vlist + cap;
        s.vcap = cap;
        if ((err = cudaMemsetAsync(s.vtotal + 1, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return err;
        int nsm = 0, dev = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
        if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
        const unsigned gp = (unsigned)std::min<long long>((long long)nsm * 8, (long long)gl);  // a few CTAs per SM
        k_vlist_fill<IdT><<<gp, kThreads, 0, st>>>(L, x, s.score, s.Cp, s.vidx, s.vlist, s.plist, s.vcap, s.vtotal + 1);
        ++launched;
    }
    if (launched_out) *launched_out = launched;
    if ((err = cudaMemsetAsync(done, 0, (size_t)L.E, st)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(s.hist, 0, sizeof(unsigned long long) * 256 * (size_t)L.E, st)) != cudaSuccess)
        return err;
    const unsigned gv = grid_for((long long)total, kThreads);
    const unsigned gw = grid_for((long long)L.E * 32, kThreads);  // a warp per (possibly) violated edge
    for (int pass = 0; pass < 8; ++pass) {
        k_select_hist_list<<<gv, kThreads, 0, st>>>(s.vlist, total, L.E, done, s.prefix, s.hist, pass);
        k_select_pick<<<gw, kThreads, 0, st>>>(s.nviol, s.hist, s.prefix, s.rem, done, pass);
    }
    k_edge_trim_list<<<gv, kThreads, 0, st>>>(s.plist, s.vtotal + 2, s.vlist, s.vcap, L.E, x, s.prefix, s.rem, done);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project(const Layout& L, float* x, double alpha, double scale, ProjScratch& s,
                           cudaStream_t st, int* launched) {
    if (L.id_bytes == 2) return project_t<uint16_t>(L, x, alpha, scale, s, st, launched);
    return project_t<int32_t>(L, x, alpha, scale, s, st, launched);
}

cudaError_t launch_project_scale(const Layout& L, float* x, const ProjScratch& s, cudaStream_t st) {
    if (L.id_bytes == 2) return project_scale_t<uint16_t>(L, x, s, st);
    return project_scale_t<int32_t>(L, x, s, st);
}

cudaError_t launch_to_user(const Layout& L, const float* x, float* out, float scale, cudaStream_t st) {
    k_to_user<<<grid_for(L.nslots * kLanes, kThreads), kThreads, 0, st>>>(L, x, out, scale);
    return cudaGetLastError();
}

cudaError_t launch_from_user(const Layout& L, const float* in, float* x, float inv_scale, cudaStream_t st) {
    k_from_user<<<grid_for(L.nslots * kLanes, kThreads), kThreads, 0, st>>>(L, in, x, inv_scale);
    return cudaGetLastError();
}

}  // namespace te

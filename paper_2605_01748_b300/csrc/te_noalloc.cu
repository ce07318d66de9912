// te_gap_noalloc: the duality gap of a caller-supplied allocation, computed
// without allocating any memory.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// want the gap -- code running inside a memory pool or arena that owns all
// device memory, a real-time control loop whose allocations are frozen after
// start-up, or a host that forbids driver allocations on its serving path.
// They pass every input and output as device pointers they already own; the
// only working memory is a fixed static device array that the library
// reserves when it is loaded.
//
// Scratch: kGapScratchSlots per-CTA partial sums (two doubles each, 256 KB),
// a file-scope __device__ array.  Every GPU on which the library is loaded
// holds it until the process exits.  Each call writes one slot per CTA it
// launches and then reads those same slots back, so nothing has to start at
// zero; but all calls on a device share the one array, so calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// and must be serialised by the caller.
#include <math.h>
#include <stdint.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "te.h"

namespace {

constexpr int kGapThreads = 256;
constexpr int kGapScratchSlots = 16384;  // demand CTAs + edge CTAs per call

static __device__ __align__(256) double g_gap_scratch[2 * kGapScratchSlots];

// Host-side device addresses of g_gap_scratch, one per device, each tagged
// with the unique id of the CUDA context it was resolved in.  After a
// cudaDeviceReset (or any re-creation of the primary context) the module is
// loaded again, possibly at another address; the id then differs and the
// address is looked up again.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    double* ptr;
};
std::mutex g_mu;
ScratchEntry g_scratch[kMaxDevices] = {};

__device__ double na_utility(double S, double alpha) {
    if (alpha == 1.0) return log(S);
    return (pow(S, 1.0 - alpha) - 1.0) / (1.0 - alpha);
}

// max over 0 <= S <= D of U_alpha(S) - pi S
__device__ double na_conj(double D, double pi, double alpha) {
    double S;
    if (alpha == 0.0) S = pi < 1.0 ? D : 0.0;
    else if (pi <= 0.0) S = D;
    else S = fmin(D, exp(-log(pi) / alpha));
    if (S <= 0.0) return na_utility(0.0, alpha);
    return na_utility(S, alpha) - pi * S;
}

// CTAs [0, ndc) take demands (primal utility and dual demand term); CTAs
// [ndc, ndc + nec) take edges (dual edge term sum p_e C_e).  Each CTA writes
// its two partial sums to scratch slot blockIdx.x.
__global__ void k_gap_partials(int K, int E, const int64_t* dpo, const int64_t* peo, const int32_t* pe,
                               const double* D, const double* C, const float* x, const double* p, double alpha,
                               int ndc, double* scratch) {
    __shared__ double red[2][kGapThreads / 32];
    double a = 0.0, b = 0.0;
    if ((int)blockIdx.x < ndc) {
        const long long c = (long long)blockIdx.x * kGapThreads + threadIdx.x;
        if (c < K) {
            double S = 0.0, pi = INFINITY;
            for (int64_t r = dpo[c]; r < dpo[c + 1]; ++r) {
                S += (double)x[r];
                double q = 0.0;
                for (int64_t i = peo[r]; i < peo[r + 1]; ++i) q += p[pe[i]];
                pi = fmin(pi, q);
            }
            a = na_utility(S, alpha);
            b = na_conj(D[c], pi, alpha);
        }
    } else {
        const long long e = (long long)(blockIdx.x - ndc) * kGapThreads + threadIdx.x;
        if (e < E) b = p[e] * C[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < kGapThreads / 32; ++i) { sa += red[0][i]; sb += red[1][i]; }
        scratch[2 * blockIdx.x] = sa;
        scratch[2 * blockIdx.x + 1] = sb;
    }
}

// One CTA sums the n partial slots in a fixed order: out = {gap, primal, dual}.
__global__ void k_gap_finish(int n, const double* scratch, double* out) {
    __shared__ double red[2][kGapThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += kGapThreads) {
        a += scratch[2 * i];
        b += scratch[2 * i + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = kGapThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[1][0] - red[0][0];
        out[1] = red[0][0];
        out[2] = red[1][0];
    }
}

// Unique id of the current context (0 if none is current or the driver
// entry points are unavailable).  The driver functions are reached through
// the runtime's entry-point query, so the library does not link libcuda.
unsigned long long current_ctx_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    if (!get_current || !get_id) return 0ull;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0ull;
    unsigned long long id = 0ull;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0ull;
    return id;
}

// Device address of g_gap_scratch on the current device, valid in the
// current context.  Resolved by cudaGetSymbolAddress (with this device
// current) on the first call per device, and again whenever the current
// context is not the one the cached address belongs to.
te_status scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TE_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchEntry& ent = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (ent.ptr && id != 0ull && ent.ctx_id == id) {
        *out = ent.ptr;
        return TE_OK;
    }
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_gap_scratch) != cudaSuccess || !ptr) return TE_ECUDA;
    // the lookup made the device's primary context current if none was
    ent.ctx_id = current_ctx_id();
    ent.ptr = static_cast<double*>(ptr);
    *out = ent.ptr;
    return TE_OK;
}

}  // namespace

extern "C" te_status te_gap_noalloc(int32_t n_edges, int32_t n_demands, int64_t n_paths, int64_t nnz,
                                    const int64_t* demand_path_off, const int64_t* path_edge_off,
                                    const int32_t* path_edges, const double* demands, const double* capacities,
                                    const float* x, const double* prices, double alpha, double* out,
                                    void* cuda_stream) {
    if (n_edges <= 0 || n_demands <= 0 || n_paths < n_demands || nnz < n_paths || !demand_path_off ||
        !path_edge_off || !path_edges || !demands || !capacities || !x || !prices || !out || !(alpha >= 0.0))
        return TE_EINVAL;
    const long long ndc = ((long long)n_demands + kGapThreads - 1) / kGapThreads;
    const long long nec = ((long long)n_edges + kGapThreads - 1) / kGapThreads;
    if (ndc + nec > kGapScratchSlots) return TE_EUNSUPPORTED;  // more than ~4.19M demands plus edges
    // an error left pending by an earlier, unrelated call is not ours to
    // clear: report it without queuing work and leave it pending
    if (cudaPeekAtLastError() != cudaSuccess) return TE_ECUDA;
    double* scratch = nullptr;
    te_status st = scratch_for_current_device(&scratch);
    if (st != TE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_gap_partials<<<(unsigned)(ndc + nec), kGapThreads, 0, s>>>(n_demands, n_edges, demand_path_off,
                                                                  path_edge_off, path_edges, demands, capacities,
                                                                  x, prices, alpha, (int)ndc, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();  // this launch's own error
        return TE_ECUDA;
    }
    k_gap_finish<<<1, kGapThreads, 0, s>>>((int)(ndc + nec), scratch, out);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return TE_ECUDA;
    }
    return TE_OK;
}

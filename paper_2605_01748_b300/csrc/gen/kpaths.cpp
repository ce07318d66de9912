// Seeded synthetic-instance helper: k hop-shortest loopless paths from every
// source to every destination of a directed graph.
//
// This file is input generation only.  It holds none of the traffic-
// engineering arithmetic: it produces the pre-computed path sets P_st that the
// TE formulation takes as an input (Section 3.1, "Variables"; the evaluation
// uses k-shortest paths, Section 4.2 "TE Inputs").
//
// Method: per source s, a layered breadth-first label-setting search.  Every
// node keeps at most k labels (partial paths from s); a label at hop h is
// extended along the node's out-edges in ascending neighbour order, a
// candidate that would revisit a node already on its path is rejected, and a
// node that already holds k labels accepts no more.  Labels are created in
// non-decreasing hop order, so each destination's labels are its k
// hop-shortest loopless paths among those whose prefixes survived the k-label
// cap (exact whenever no needed prefix was pruned; an approximation of Yen's
// algorithm otherwise).  Ties are broken by creation order, which is
// deterministic.  Sources are processed in parallel with OpenMP; the output
// order is (source, destination, label) and does not depend on the thread
// count.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Label {
    int32_t node;
    int32_t parent;  // index of the parent label, -1 for the root
    int32_t edge;    // edge id used to reach `node`
    int32_t hops;
};

struct SourceResult {
    std::vector<int32_t> dst;          // destination of each demand (pair)
    std::vector<int32_t> npaths;       // paths per demand
    std::vector<int32_t> path_len;     // hops per path
    std::vector<int32_t> edges;        // concatenated edge ids
};

struct Result {
    int64_t n_demands = 0, n_paths = 0, nnz = 0;
    std::vector<SourceResult> per_source;
};

void run_source(int s, int n, const int64_t* adj_off, const int32_t* adj_dst,
                const int32_t* adj_eid, int k, int max_hops, SourceResult& out) {
    std::vector<Label> L;
    L.reserve((size_t)n * (size_t)k / 2 + 16);
    std::vector<int32_t> cnt(n, 0);
    cnt[s] = k;  // a loopless path never returns to its source
    L.push_back({s, -1, -1, 0});
    size_t head = 0;
    while (head < L.size()) {
        size_t end = L.size();
        for (; head < end; ++head) {
            const Label cur = L[head];
            if (cur.hops >= max_hops) continue;
            for (int64_t j = adj_off[cur.node]; j < adj_off[cur.node + 1]; ++j) {
                const int32_t w = adj_dst[j];
                if (cnt[w] >= k) continue;
                bool loop = false;
                for (int32_t p = (int32_t)head; p != -1; p = L[p].parent) {
                    if (L[p].node == w) { loop = true; break; }
                }
                if (loop) continue;
                L.push_back({w, (int32_t)head, adj_eid[j], cur.hops + 1});
                cnt[w]++;
            }
        }
    }
    // bucket labels by destination, preserving creation order
    std::vector<int32_t> first(n + 1, 0);
    for (size_t i = 1; i < L.size(); ++i) first[L[i].node + 1]++;
    for (int v = 0; v < n; ++v) first[v + 1] += first[v];
    std::vector<int32_t> order(L.size() > 0 ? L.size() - 1 : 0);
    std::vector<int32_t> fill(first.begin(), first.end() - 1);
    for (size_t i = 1; i < L.size(); ++i) order[fill[L[i].node]++] = (int32_t)i;
    std::vector<int32_t> tmp;
    for (int t = 0; t < n; ++t) {
        if (t == s) continue;
        const int32_t c = first[t + 1] - first[t];
        if (c == 0) continue;
        out.dst.push_back(t);
        out.npaths.push_back(c);
        for (int32_t q = first[t]; q < first[t + 1]; ++q) {
            tmp.clear();
            for (int32_t p = order[q]; L[p].parent != -1; p = L[p].parent) tmp.push_back(L[p].edge);
            out.path_len.push_back((int32_t)tmp.size());
            for (size_t h = tmp.size(); h-- > 0;) out.edges.push_back(tmp[h]);
        }
    }
}

}  // namespace

extern "C" {

// Computes the path sets.  adj_off[n+1], adj_dst[m], adj_eid[m] is the
// out-adjacency in CSR form (neighbours sorted ascending by the caller).
// Returns 0 on success and a handle that tegen_fetch/tegen_free consume;
// counts[0..2] = demands (pairs with at least one path), paths, nonzeros.
int tegen_kpaths(int n, const int64_t* adj_off, const int32_t* adj_dst, const int32_t* adj_eid,
                 int k, int max_hops, int nthreads, void** handle, int64_t* counts) {
    if (n <= 0 || k <= 0 || !adj_off || !adj_dst || !adj_eid || !handle || !counts) return 1;
    Result* R = new Result();
    R->per_source.resize(n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < n; ++s) run_source(s, n, adj_off, adj_dst, adj_eid, k, max_hops, R->per_source[s]);
    for (int s = 0; s < n; ++s) {
        R->n_demands += (int64_t)R->per_source[s].dst.size();
        R->n_paths += (int64_t)R->per_source[s].path_len.size();
        R->nnz += (int64_t)R->per_source[s].edges.size();
    }
    counts[0] = R->n_demands;
    counts[1] = R->n_paths;
    counts[2] = R->nnz;
    *handle = R;
    return 0;
}

// Copies the result into caller-allocated arrays: dsrc/ddst[n_demands],
// dpo[n_demands+1], peo[n_paths+1], pe[nnz].
int tegen_fetch(void* handle, int32_t* dsrc, int32_t* ddst, int64_t* dpo, int64_t* peo, int32_t* pe) {
    Result* R = (Result*)handle;
    if (!R) return 1;
    const int n = (int)R->per_source.size();
    std::vector<int64_t> dbase(n + 1, 0), pbase(n + 1, 0), ebase(n + 1, 0);
    for (int s = 0; s < n; ++s) {
        dbase[s + 1] = dbase[s] + (int64_t)R->per_source[s].dst.size();
        pbase[s + 1] = pbase[s] + (int64_t)R->per_source[s].path_len.size();
        ebase[s + 1] = ebase[s] + (int64_t)R->per_source[s].edges.size();
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int s = 0; s < n; ++s) {
        const SourceResult& S = R->per_source[s];
        int64_t d = dbase[s], p = pbase[s], e = ebase[s];
        std::memcpy(pe + e, S.edges.data(), S.edges.size() * sizeof(int32_t));
        size_t q = 0;
        for (size_t i = 0; i < S.dst.size(); ++i, ++d) {
            dsrc[d] = s;
            ddst[d] = S.dst[i];
            dpo[d] = p;
            for (int32_t j = 0; j < S.npaths[i]; ++j, ++q, ++p) {
                peo[p] = e;
                e += S.path_len[q];
            }
        }
    }
    dpo[R->n_demands] = R->n_paths;
    peo[R->n_paths] = R->nnz;
    return 0;
}

void tegen_free(void* handle) { delete (Result*)handle; }

}  // extern "C"

// Host-side construction of the sliced device layout (see te_layout.h and
// the layout description in te_internal.cuh).
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "te_banks.h"
#include "te_layout.h"

namespace te {
namespace {

std::string fmt(const char* f, long long a, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

}  // namespace

te_status build_host_layout(const te_topology* topo, const te_paths* P, const double* D, const double* C,
                            double scale, int g_min, HostLayout& out, int max_id_bytes) {
    const int E = topo->n_edges;
    const int K = P->n_demands;
    (void)C;
    // sort demands by (path count, lengths of the first 11 paths) so the 32
    // demands of a block have alike path lengths and padding stays small
    std::vector<std::pair<unsigned long long, int>> order(K);
    int kmax = 0;
    for (int c = 0; c < K; ++c) {
        const long long p0 = P->demand_path_off[c], np = P->demand_path_off[c + 1] - p0;
        kmax = std::max(kmax, (int)np);
        unsigned long long key = (unsigned long long)np << 58;
        for (int j = 0; j < 11 && j < np; ++j) {
            long long len = P->path_edge_off[p0 + j + 1] - P->path_edge_off[p0 + j];
            if (len > 31) len = 31;
            key |= (unsigned long long)len << (53 - 5 * j);
        }
        order[c] = {key, c};
    }
    std::sort(order.begin(), order.end());
    // lanes per demand: no lane holds more than kMaxPathsPerLane paths
    int G = g_min > 1 ? g_min : 1;
    while (G * te::kMaxPathsPerLane < kmax) G *= 2;
    const int DPB = kLanes / G;  // demands per block
    const int kl = (kmax + G - 1) / G;
    const int nblocks = (K + DPB - 1) / DPB;
    auto demand_at = [&](int b, int t) -> int {  // demand index of block b, position t, or -1
        const long long q = (long long)b * DPB + t;
        return q < K ? order[q].second : -1;
    };
    auto path_len = [&](int c, long long p) -> long long {
        const long long r = P->demand_path_off[c] + p;
        return P->path_edge_off[r + 1] - P->path_edge_off[r];
    };
    std::vector<int> slotbase(nblocks + 1, 0);
    for (int b = 0; b < nblocks; ++b) {
        int kb = 0;
        for (int t = 0; t < DPB; ++t) {
            const int c = demand_at(b, t);
            if (c < 0) break;
            const int np = (int)(P->demand_path_off[c + 1] - P->demand_path_off[c]);
            kb = std::max(kb, (np + G - 1) / G);
        }
        slotbase[b + 1] = slotbase[b] + kb;
    }
    const long long nslots = slotbase[nblocks];
    std::vector<unsigned> rowoff(nslots + 1, 0);
    std::vector<te::BlockMeta> blkmeta(nblocks);
    int max_block_rows = 0;
    for (int b = 0; b < nblocks; ++b) {
        const int kb = slotbase[b + 1] - slotbase[b];
        unsigned counts = 0;
        for (int j = 0; j < kb; ++j) {
            long long H = 0;
            for (int t = 0; t < DPB; ++t) {
                const int c = demand_at(b, t);
                if (c < 0) break;
                const long long np = P->demand_path_off[c + 1] - P->demand_path_off[c];
                for (int hh = 0; hh < G; ++hh) {
                    const long long p = (long long)j * G + hh;
                    if (p < np) H = std::max<long long>(H, path_len(c, p));
                }
            }
            const long long s = slotbase[b] + j;
            const long long next = (long long)rowoff[s] + H;
            if (next > 0xffffffffLL) { out.err = "instance too large for the 32-bit row index"; return TE_EUNSUPPORTED; }
            rowoff[s + 1] = (unsigned)next;
            counts |= (unsigned)H << (8 * j);
        }
        blkmeta[b].s0 = (unsigned)slotbase[b];
        blkmeta[b].row0 = rowoff[slotbase[b]];
        blkmeta[b].counts = counts;
        blkmeta[b].kb = (unsigned)kb;
        max_block_rows = std::max<int>(max_block_rows, (int)(rowoff[slotbase[b + 1]] - rowoff[slotbase[b]]));
    }
    const long long nrows = rowoff[nslots];
    const bool ids32 = E + 1 > 65535;
    if (ids32 && max_id_bytes < 4) {
        out.err = fmt("n_edges = %lld: this kernel takes 16-bit edge ids (at most 65534 edges)", E); return TE_EUNSUPPORTED;
    }
    out.id_bytes = ids32 ? 4 : 2;
    const size_t ND = (size_t)nblocks * DPB;  // demand slots
    if (ids32) out.ids32.assign((size_t)nrows * kLanes, (uint32_t)E);
    else out.ids.assign((size_t)nrows * kLanes, (uint16_t)E);
    std::vector<long long> slot_path((size_t)nslots * kLanes, -1);
    std::vector<unsigned> hops((size_t)nblocks * kLanes, 0u);
    std::vector<int> demand_of(ND, -1);
    std::vector<float> Dn(ND, 0.f);
    std::vector<double> Dc(ND, 0.0);
    std::vector<unsigned char> npv(ND, 0);
    for (int b = 0; b < nblocks; ++b) {
        for (int t = 0; t < DPB; ++t) {
            const int c = demand_at(b, t);
            if (c < 0) break;
            const long long p0 = P->demand_path_off[c], np = P->demand_path_off[c + 1] - p0;
            const size_t di = (size_t)b * DPB + t;
            demand_of[di] = c;
            Dn[di] = (float)(D[c] / scale);
            Dc[di] = D[c];
            npv[di] = (unsigned char)np;
            for (long long p = 0; p < np; ++p) {
                const int lane = t * G + (int)(p % G);
                const long long s = slotbase[b] + p / G, r = p0 + p;
                slot_path[(size_t)s * kLanes + lane] = r;
                const long long i0 = P->path_edge_off[r], n = P->path_edge_off[r + 1] - i0;
                hops[(size_t)b * kLanes + lane] |= (unsigned)n << (8 * (p / G));
                for (long long k = 0; k < n; ++k) {
                    const size_t at = ((size_t)rowoff[s] + (size_t)k) * kLanes + lane;
                    if (ids32) out.ids32[at] = (uint32_t)P->path_edges[i0 + k];
                    else out.ids[at] = (uint16_t)P->path_edges[i0 + k];
                }
            }
        }
    }
    // hop order within each slot: spread every row's ids over the shared-memory banks
    if (!ids32) {
        uint16_t* q = out.ids.data();
        const unsigned hw = std::thread::hardware_concurrency();
        const long long nt = std::max<long long>(1, std::min<long long>({hw ? (long long)hw : 1LL, 64LL, nslots}));
        std::vector<std::thread> pool;
        for (long long w = 0; w < nt; ++w)
            pool.emplace_back([&, w]() {
                for (long long s = w; s < nslots; s += nt)
                    te::balance_slot_banks(q + (size_t)rowoff[s] * kLanes, (int)(rowoff[s + 1] - rowoff[s]),
                                           (uint16_t)E);
            });
        for (auto& t : pool) t.join();
    }
    std::vector<float> cap_n(E), ne_f(E, 0.f), inv_ne(E, 0.f);
    {
        std::vector<long long> ne(E, 0);
        for (long long i = 0; i < P->nnz; ++i) ne[P->path_edges[i]]++;
        for (int e = 0; e < E; ++e) {
            cap_n[e] = (float)(C[e] / scale);
            ne_f[e] = (float)ne[e];
            inv_ne[e] = ne[e] > 0 ? (float)(1.0 / (double)ne[e]) : 0.f;
        }
        // range of the kernel's 32-bit fixed-point load histograms: a rate
        // adds floor(x 2^12) and a remainder below 2^12 (units of 2^-24), and
        // the rates of a demand sum to at most D_c, so every per-CTA sum stays
        // below 2^32 when each edge has fewer than 2^19 paths and the demands
        // with a path through it total less than 2^19 (normalised)
        std::vector<double> dsum(E, 0.0);
        std::vector<int> stamp(E, -1);
        for (int c = 0; c < K; ++c) {
            const double d = D[c] / scale;
            for (long long i = P->path_edge_off[P->demand_path_off[c]]; i < P->path_edge_off[P->demand_path_off[c + 1]]; ++i) {
                const int e = P->path_edges[i];
                if (stamp[e] != c) { stamp[e] = c; dsum[e] += d; }
            }
        }
        for (int e = 0; e < E; ++e)
            if (ne[e] >= (1LL << 19) || dsum[e] >= (double)(1 << 19)) {
                out.err = fmt("edge %lld: %lld paths, or the demands with a path through it, exceed the range of the "
                             "load histograms (2^19 paths, 2^19 in normalised demand)", e, ne[e]); return TE_EUNSUPPORTED;
            }
    }


    out.E = E;
    out.K = K;
    out.P = P->n_paths;
    out.nnz = P->nnz;
    out.G = G;
    out.dpb = DPB;
    out.kl = kl;
    out.kmax = kmax;
    out.nblocks = nblocks;
    out.max_block_rows = max_block_rows;
    out.nslots = nslots;
    out.nrows = nrows;
    out.rowoff = std::move(rowoff);
    out.slotbase = std::move(slotbase);
    out.blkmeta = std::move(blkmeta);
    out.hops = std::move(hops);
    out.demand_of = std::move(demand_of);
    out.Dn = std::move(Dn);
    out.Dc = std::move(Dc);
    out.np = std::move(npv);
    out.slot_path = std::move(slot_path);
    out.cap_n = std::move(cap_n);
    out.ne_f = std::move(ne_f);
    out.inv_ne = std::move(inv_ne);
    return TE_OK;
}

}  // namespace te

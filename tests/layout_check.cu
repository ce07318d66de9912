// Host-only check of the sliced layout that te_create builds (te_layout.cu),
// compiled and run by tests/test_layout_host.py on a machine without a GPU.
//
// usage: layout_check <dir>
// <dir> holds the instance as raw little-endian arrays: esrc.bin, edst.bin
// (int32 [E]), cap.bin (float64 [E]), dem.bin (float64 [K]), dpo.bin
// (int64 [K+1]), peo.bin (int64 [P+1]), pe.bin (int32 [nnz]).  Prints
// "OK ..." and exits 0 when every property holds, else "FAIL ..." and exits 1.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "te_layout.h"

template <class T>
static std::vector<T> read_all(const char* dir, const char* name) {
    char path[1024];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE* f = fopen(path, "rb");
    if (!f) {
        printf("FAIL cannot open %s\n", path);
        exit(1);
    }
    fseek(f, 0, SEEK_END);
    const long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    std::vector<T> v((size_t)n / sizeof(T));
    if (fread(v.data(), 1, (size_t)n, f) != (size_t)n) {
        printf("FAIL short read of %s\n", path);
        exit(1);
    }
    fclose(f);
    return v;
}

#define CHECK(cond, ...)              \
    do {                              \
        if (!(cond)) {                \
            printf("FAIL ");          \
            printf(__VA_ARGS__);      \
            printf("\n");             \
            return 1;                 \
        }                             \
    } while (0)

int main(int argc, char** argv) {
    if (argc < 2) {
        printf("FAIL usage: layout_check <dir>\n");
        return 1;
    }
    const char* dir = argv[1];
    auto es = read_all<int32_t>(dir, "esrc.bin");
    auto ed = read_all<int32_t>(dir, "edst.bin");
    auto cap = read_all<double>(dir, "cap.bin");
    auto dem = read_all<double>(dir, "dem.bin");
    auto dpo = read_all<int64_t>(dir, "dpo.bin");
    auto peo = read_all<int64_t>(dir, "peo.bin");
    auto pe = read_all<int32_t>(dir, "pe.bin");
    const int E = (int)cap.size();
    const int K = (int)dem.size();
    te_topology topo{0, E, es.data(), ed.data()};
    te_paths P{};
    P.n_demands = K;
    P.n_paths = (int64_t)peo.size() - 1;
    P.nnz = (int64_t)pe.size();
    P.demand_path_off = dpo.data();
    P.path_edge_off = peo.data();
    P.path_edges = pe.data();
    te::HostLayout L;
    // 32-bit ids allowed (taken only above 65,534 edges)
    const te_status st = te::build_host_layout(&topo, &P, dem.data(), cap.data(), 1.0, 1, L, 4);
    CHECK(st == TE_OK, "build_host_layout returned %d: %s", (int)st, L.err.c_str());

    const int G = L.G, DPB = L.dpb;
    CHECK(G * DPB == te::kLanes, "G %d x demands per block %d != 32", G, DPB);
    CHECK((long long)L.rowoff.size() == L.nslots + 1 && L.rowoff[0] == 0, "row offsets");
    const bool ids32 = L.id_bytes == 4;
    CHECK(ids32 == (E > 65534) && (L.id_bytes == 2 || ids32), "id width %d for %d edges", L.id_bytes, E);
    CHECK((long long)(ids32 ? L.ids32.size() : L.ids.size()) == L.nrows * te::kLanes, "id array size");
    auto id_of = [&](size_t at) -> long long { return ids32 ? (long long)L.ids32[at] : (long long)L.ids[at]; };
    CHECK((int)L.hops.size() == L.nblocks * te::kLanes, "hop-count array size");
    std::vector<int> seen(K, 0);
    long long pad = 0, paths_seen = 0;
    for (int b = 0; b < L.nblocks; ++b) {
        const int s0 = L.slotbase[b], kb = L.slotbase[b + 1] - s0;
        const te::BlockMeta& m = L.blkmeta[b];
        CHECK((int)m.s0 == s0 && (int)m.kb == kb && m.row0 == L.rowoff[s0], "block %d record", b);
        CHECK(kb >= 1 && kb <= te::kMaxPathsPerLane, "block %d has %d slots", b, kb);
        for (int j = 0; j < te::kMaxPathsPerLane; ++j) {
            const unsigned rows = j < kb ? L.rowoff[s0 + j + 1] - L.rowoff[s0 + j] : 0u;
            CHECK(((m.counts >> (8 * j)) & 0xffu) == rows, "block %d slot %d row count", b, j);
        }
        for (int t = 0; t < DPB; ++t) {
            const size_t di = (size_t)b * DPB + t;
            const int c = L.demand_of[di];
            const int np = L.np[di];
            if (c < 0) {
                CHECK(np == 0, "padding demand slot %zu has paths", di);
                continue;
            }
            CHECK(c < K && seen[c] == 0, "demand %d placed twice or out of range", c);
            seen[c] = 1;
            CHECK(np == (int)(dpo[c + 1] - dpo[c]), "demand %d path count", c);
            CHECK(L.Dc[di] == dem[c], "demand %d value", c);
        }
        for (int lane = 0; lane < te::kLanes; ++lane) {
            const unsigned hops = L.hops[(size_t)b * te::kLanes + lane];
            for (int j = 0; j < te::kMaxPathsPerLane; ++j) {
                const unsigned n_j = (hops >> (8 * j)) & 0xffu;
                if (j >= kb) {
                    CHECK(n_j == 0, "block %d lane %d: hop count in a missing slot", b, lane);
                    continue;
                }
                const size_t s = (size_t)s0 + j;
                const long long r = L.slot_path[s * te::kLanes + lane];
                std::vector<int> got;
                for (unsigned row = L.rowoff[s]; row < L.rowoff[s + 1]; ++row) {
                    const int id = (int)id_of((size_t)row * te::kLanes + lane);
                    if (id == E) {
                        ++pad;
                        continue;
                    }
                    CHECK(id >= 0 && id < E, "slot %zu lane %d: id %d out of range", s, lane, id);
                    got.push_back(id);
                }
                std::vector<int> want;
                if (r >= 0) {
                    ++paths_seen;
                    // the path belongs to this lane's demand, as path j*G + lane%G
                    const int c = L.demand_of[(size_t)b * DPB + lane / G];
                    CHECK(c >= 0 && r == dpo[c] + (long long)j * G + lane % G, "slot %zu lane %d: path %lld", s,
                          lane, r);
                    for (long long i = peo[r]; i < peo[r + 1]; ++i) want.push_back(pe[i]);
                }
                CHECK(n_j == want.size(), "block %d lane %d slot %d: hop count %u, path has %zu edges", b, lane, j,
                      n_j, want.size());
                std::sort(got.begin(), got.end());
                std::sort(want.begin(), want.end());
                CHECK(got == want, "slot %zu lane %d: the ids are not the path's edges", s, lane);
            }
        }
    }
    for (int c = 0; c < K; ++c) CHECK(seen[c] == 1, "demand %d missing from the layout", c);
    CHECK(paths_seen == P.n_paths, "%lld paths in the layout, %lld in the instance", paths_seen,
          (long long)P.n_paths);
    CHECK(pad + P.nnz == L.nrows * te::kLanes, "padding count");
    printf("OK G=%d blocks=%d slots=%lld rows=%lld padding=%lld\n", G, L.nblocks, L.nslots, L.nrows, pad);
    return 0;
}

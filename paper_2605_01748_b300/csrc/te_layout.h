// Host-side construction of the sliced device layout of one instance (the
// arrays the iteration kernel and the projection read), shared by the
// single-instance handle and the batch.  Declarations only; see te_layout.cu.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "te.h"
#include "te_internal.cuh"

namespace te {

struct HostLayout {
    int E = 0, K = 0;
    long long P = 0, nnz = 0;
    int G = 1, dpb = 32, kl = 0, kmax = 0, nblocks = 0, max_block_rows = 0;
    long long nslots = 0, nrows = 0;
    int id_bytes = 2;                    // 2: ids below, 4: ids32 (more than 65,534 edges)
    std::vector<uint16_t> ids;           // [nrows*32] (id_bytes 2)
    std::vector<uint32_t> ids32;         // [nrows*32] (id_bytes 4)
    std::vector<unsigned> rowoff;        // [nslots+1]
    std::vector<int> slotbase;           // [nblocks+1]
    std::vector<BlockMeta> blkmeta;      // [nblocks]
    std::vector<unsigned> hops;          // [nblocks*32] hop counts of a lane's paths, slot j in bits 8j..8j+7
    std::vector<int> demand_of;          // [nblocks*dpb]
    std::vector<float> Dn;               // [nblocks*dpb]
    std::vector<double> Dc;              // [nblocks*dpb]
    std::vector<unsigned char> np;       // [nblocks*dpb]
    std::vector<long long> slot_path;    // [nslots*32]
    std::vector<float> cap_n, ne_f, inv_ne;  // [E]
    std::string err;
};

// Builds the layout of an instance already checked for validity: demands
// sorted by their path lengths into blocks of 32/G demands (G >= g_min lanes
// per demand, at most kMaxPathsPerLane paths per lane), each path's hops
// ordered within its slot to spread every row over the shared-memory banks,
// values normalised by scale.  Edge ids are 16-bit, or 32-bit (hops in path
// order, no bank order: only the wide-edge mode reads them, from global
// memory) when there are more than 65,534 edges and max_id_bytes is 4.
// Returns TE_OK, or TE_EUNSUPPORTED with err set.
te_status build_host_layout(const te_topology* topo, const te_paths* P, const double* D, const double* C,
                            double scale, int g_min, HostLayout& out, int max_id_bytes = 2);

}  // namespace te

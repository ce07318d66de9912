// Host-side layout helper: bank-aware hop order within one slot.
//
// The iteration kernel reads w[id] and adds into the histogram h[id] for the
// 32 ids of one row of a slot at a time (one warp-wide shared-memory access
// each).  32-bit words in shared memory fall into bank id % 32, and lanes
// whose ids share a bank (or the same id) are served one after another.  The
// sums the kernels form over a path's edges do not depend on the order of its
// hops, so each lane's edges may be placed in any rows of its slot.  This
// reorders them greedily, row by row: a lane that must place an edge in this
// row (as many edges left as rows) takes the edge of its least-loaded bank;
// a lane with rows to spare places an edge only into a bank nobody in the
// row has used yet, else it leaves a padding entry (the sentinel id) for a
// later row.
#pragma once

#include <stdint.h>

namespace te {

inline void balance_slot_banks(uint16_t* rows, int H, uint16_t sentinel) {
    constexpr int kL = 32;
    if (H <= 1) return;
    uint16_t left[kL][256];
    int n[kL];
    for (int l = 0; l < kL; ++l) {
        n[l] = 0;
        for (int r = 0; r < H; ++r) {
            const uint16_t id = rows[r * kL + l];
            if (id != sentinel) left[l][n[l]++] = id;
        }
    }
    for (int r = 0; r < H; ++r) {
        const int rows_left = H - r;
        int cnt[kL] = {0};
        uint16_t out[kL];
        for (int l = 0; l < kL; ++l) out[l] = sentinel;
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < kL; ++l) {
                if (n[l] == 0 || out[l] != sentinel) continue;  // nothing left, or placed in pass 0
                const bool forced = n[l] >= rows_left;
                if (forced != (pass == 0)) continue;
                int best = 0, bc = 1 << 30;
                for (int k = 0; k < n[l]; ++k) {
                    const int c = cnt[left[l][k] % kL];
                    if (c < bc) { bc = c; best = k; }
                }
                if (!forced && bc > 0) continue;  // wait for a freer row
                out[l] = left[l][best];
                cnt[out[l] % kL]++;
                left[l][best] = left[l][--n[l]];
            }
        }
        for (int l = 0; l < kL; ++l) rows[r * kL + l] = out[l];
    }
}

}  // namespace te

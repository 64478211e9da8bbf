// The launch plan of one subsequence search, shared by subseq_search and
// subseq_search_noalloc: which wavefront runs each level, and the slots of the
// search's small integer state array.
#pragma once

#include <cstdint>

#include "dtw_elastic.cuh"

namespace eapdtw {

constexpr int kMaxLevels = 4;   // levels 0..kMaxLevels (at most five: K = 4, 8, 16, 32, group)

// Work levels: the first launch runs every window; windows whose live region
// overflowed the previous level's window of blocks are re-run by the next one,
// up to the widest (a group of warps holding every column).
struct Plan {
    int nlev = 0;
    int K[kMaxLevels + 1];
    int band[kMaxLevels + 1];
    bool wide[kMaxLevels + 1];      // a group of warps per candidate (dtw_group.cuh): the widest level,
                                    // or the first one (with the lower bounds) when the tile hint asks
    bool elastic[kMaxLevels + 1];   // the narrow-block elastic wavefront (unconstrained first level)
};

// Tile hint that makes the first level a group of warps (any query length).
constexpr int kGroupTileHint = 512;
// Bands that start on the elastic wavefront: w >= kElBandMinW and w >= nc x
// kElBandMinQuarters / 4 (compile-time knobs for tuning experiments).
#ifndef EAPDTW_ELASTIC_BAND_MIN_W
#define EAPDTW_ELASTIC_BAND_MIN_W 64
#endif
#ifndef EAPDTW_ELASTIC_BAND_MIN_QUARTERS
#define EAPDTW_ELASTIC_BAND_MIN_QUARTERS 1
#endif
constexpr int kElBandMinW = EAPDTW_ELASTIC_BAND_MIN_W;
constexpr int kElBandMinQuarters = EAPDTW_ELASTIC_BAND_MIN_QUARTERS;

// nr, nc: rows and columns of the DP (window and query lengths); w: the window
// (w >= max(nr, nc) - 1 is unconstrained); tile_hint: 4, 8, 16 or 32 fixes the
// first level's K, kGroupTileHint makes it a group of warps, 0 chooses.
// search_levels: the first level may be the elastic wavefront (unconstrained,
// or, for queries of up to 1024 points, a band of at least kElBandMinW and a
// quarter of the query: longer ones come with wider live regions that it
// mostly hands over) or, on
// request, a group of warps; neither implements upper-bound tightening, and
// the pair kernel has neither.
inline Plan plan_levels(int64_t nr, int64_t nc, int64_t w, int tile_hint, bool search_levels = true) {
    const int64_t lmax = nr > nc ? nr : nc;
    const bool unconstrained = w >= lmax - 1;
    Plan p;
    int covered = 0;  // columns of the widest window of the previous level
    int k0 = 32;
    if (tile_hint == 4 || tile_hint == 8 || tile_hint == 16 || tile_hint == 32) {
        k0 = tile_hint;
    } else if (search_levels && tile_hint == kGroupTileHint && nc <= 8 * 512) {
        p.K[0] = 16;
        p.band[0] = unconstrained ? 0 : (16 <= 2 * w + 2 ? 1 : 2);
        p.wide[0] = true;
        p.elastic[0] = false;
        p.nlev = 1;
        return p;
    } else if (!unconstrained) {
        // blocks spanned by the band across the pipelined rows, plus margin;
        // no wider than needed for one window to hold every column (then
        // nothing can overflow it)
        for (int K = 4; K <= 32; K *= 2)
            if ((2 * w + K) / (K + 1) + 3 <= 32 || 32 * K >= nc) { k0 = K; break; }
        // A wide band: the elastic wavefront first, handing the candidates
        // whose live region nears the band's edges (or outgrows its windows)
        // to the banded levels below.
        if (search_levels && nc > 32 * 4 && nc <= 32 * 32 && w >= kElBandMinW && 4 * w >= kElBandMinQuarters * nc) {
            p.K[0] = kElK;
            p.band[0] = 1;
            p.wide[0] = false;
            p.elastic[0] = true;
            p.nlev = 1;
        }
        // A band that fits no warp's window still starts with one warp at
        // K = 32: measured on GB300 a group of warps as the first level was
        // slower (its warps wait on one another while the live region is
        // narrower than the band), so the group only re-runs the overflows.
    } else if (search_levels && nc > 32 * 4) {
        p.K[0] = kElK;
        p.band[0] = 0;
        p.wide[0] = false;
        p.elastic[0] = true;
        p.nlev = 1;
        covered = 32 * kElJ * kElK;
        k0 = 8;
    } else {
        k0 = 8;
        for (int K = 4; K <= 8; K *= 2)
            if (32 * K >= nc) { k0 = K; break; }
    }
    for (int K = k0; K <= 32; K *= 2) {
        const int band = unconstrained ? 0 : (K <= 2 * w + 2 ? 1 : 2);
        const int cols = 32 * K * dtw_windows(K, band);
        if (cols <= covered) continue;
        p.K[p.nlev] = K;
        p.band[p.nlev] = band;
        p.wide[p.nlev] = false;
        p.elastic[p.nlev] = false;
        ++p.nlev;
        covered = cols;
    }
    // Last level: a group of warps of blocks of 16 columns (up to 4096
    // columns; the pair kernel's widest level: K = 32 with the columns
    // streamed), needed only when the columns do not fit one window of K = 32
    // (an empty re-run list makes it a no-op launch).
    if (nc > 32 * 32) {
        const int kw = search_levels ? 16 : 32;
        p.K[p.nlev] = kw;
        p.band[p.nlev] = unconstrained ? 0 : (kw <= 2 * w + 2 ? 1 : 2);
        p.wide[p.nlev] = true;
        p.elastic[p.nlev] = false;
        ++p.nlev;
    }
    return p;
}

// Slots of the search's int array (device).
enum IntSlot : int {
    kWork0 = 0,                             // work counters of levels 0..kMaxLevels
    kWorkSeed = kWork0 + kMaxLevels + 1,
    kOvf0 = kWorkSeed + 1,                  // overflow counts written by levels 0..kMaxLevels
    kBad = kOvf0 + kMaxLevels + 1,
    kNBest = kBad + 1,
    kSeedOvf = kNBest + 1,
    kWorkTail = kSeedOvf + 1,               // probe: entries of the sample list; kWorkTail + 1: its work counter
    kProbeCount = kWorkTail + 2,            // overflows among the probe's windows
    kTimeout = kProbeCount + 1,             // 1: a device-side wait of the group level ran out
    kDbgSlot = 24,                          // 24.. hold the device self-check record
    kNumInts = 32
};
static_assert(kTimeout < kDbgSlot, "int slots overlap the device self-check record");

}  // namespace eapdtw

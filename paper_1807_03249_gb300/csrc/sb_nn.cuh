// Exact nearest-neighbour search in a source guide (Section 3.1: the table
// lookup of u*; with more guide channels the paper retrieves u* with search
// trees instead).  The index is a two-level tree of guide-space boxes over the
// source: the per-channel min/max of every 16 x 16-pixel tile, and of every
// 4 x 4-tile super-tile.  A box whose squared distance to the query exceeds
// the best distance found so far (or equals it while its first pixel comes
// after the best pixel) cannot hold a better pixel and is skipped, so the
// result equals the brute-force argmin with ties to the smallest y * W + x.
#pragma once

#include "sb_internal.cuh"

namespace sb {

constexpr int kLutTile = 16;  // pixels per tile side
constexpr int kSuper = 4;     // tiles per super-tile side

// Boxes of a source of W x H pixels: tiles_x x tiles_y tile boxes, then the
// super-tile boxes (row-major each).  Box channel c: min | max << 16.
struct NnGeometry {
    int tiles_x, tiles_y, n_tiles, supers_x, n_supers;
    __host__ __device__ static NnGeometry of(int W, int H) {
        NnGeometry g;
        g.tiles_x = (W + kLutTile - 1) / kLutTile;
        g.tiles_y = (H + kLutTile - 1) / kLutTile;
        g.n_tiles = g.tiles_x * g.tiles_y;
        g.supers_x = (g.tiles_x + kSuper - 1) / kSuper;
        g.n_supers = g.supers_x * ((g.tiles_y + kSuper - 1) / kSuper);
        return g;
    }
};

// squared distance from a query (channel values rep[c]) to a guide box,
// over the first kc channels
template <int C, int B>
__device__ __forceinline__ uint64_t box_distance(const uint32_t (&rep)[C], uint4 bb, int kc) {
    const uint32_t w[4] = {bb.x, bb.y, bb.z, bb.w};
    uint64_t lb = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (c >= kc) break;
        const uint32_t lo = w[c] & 0xFFFFu, hi = w[c] >> 16;
        const uint32_t t = rep[c] < lo ? lo - rep[c] : (rep[c] > hi ? rep[c] - hi : 0u);
        lb += (uint64_t)t * t;
    }
    return lb;
}

// Nearest pixel of tile t to the packed query (channels from kc on zero):
// updates the best squared distance bd and its linear index bl.
template <int C, int B>
__device__ __forceinline__ void nn_scan_tile(const uint32_t *packed, int W, int H, int tiles_x,
                                             int t, uint32_t q_packed, int kc, uint64_t &bd,
                                             uint32_t &bl) {
    using F = GuideFmt<C, B>;
    const int x0 = (t % tiles_x) * kLutTile, y0 = (t / tiles_x) * kLutTile;
    const int x1 = min(x0 + kLutTile, W), y1 = min(y0 + kLutTile, H);
    for (int y = y0; y < y1; ++y) {
        for (int x = x0; x < x1; ++x) {
            const uint32_t lin = (uint32_t)y * (uint32_t)W + (uint32_t)x;
            const uint64_t d = F::dist(q_packed, F::key_part(__ldg(packed + lin), kc));
            if (d < bd || (d == bd && lin < bl)) {
                bd = d;
                bl = lin;
            }
        }
    }
}

// One thread's query: the source position (x | y << 16) whose guide is
// nearest to q over the first kc channels, ties to the smallest y * W + x.
// Start from the nearest tile of the nearest super-tile, then visit every
// box that could still hold a better or tied-earlier pixel.
template <int C, int B>
__device__ __noinline__ uint32_t nn_query(const uint32_t *packed, const uint4 *bounds, int W, int H,
                                          uint32_t q_packed, int kc) {
    using F = GuideFmt<C, B>;
    const NnGeometry g = NnGeometry::of(W, H);
    uint32_t rep[C];
#pragma unroll
    for (int c = 0; c < C; ++c) rep[c] = F::chan(q_packed, c);
    const uint4 *sup = bounds + g.n_tiles;
    uint64_t best_lb = ~0ull;
    int best_s = 0;
    for (int st = 0; st < g.n_supers; ++st) {
        const uint64_t lb = box_distance<C, B>(rep, __ldg(&sup[st]), kc);
        if (lb < best_lb) {
            best_lb = lb;
            best_s = st;
        }
    }
    const int stx0 = (best_s % g.supers_x) * kSuper, sty0 = (best_s / g.supers_x) * kSuper;
    int best_t = sty0 * g.tiles_x + stx0;
    best_lb = ~0ull;
    for (int ty = sty0; ty < min(sty0 + kSuper, g.tiles_y); ++ty)
        for (int tx = stx0; tx < min(stx0 + kSuper, g.tiles_x); ++tx) {
            const uint64_t lb = box_distance<C, B>(rep, __ldg(&bounds[ty * g.tiles_x + tx]), kc);
            if (lb < best_lb) {
                best_lb = lb;
                best_t = ty * g.tiles_x + tx;
            }
        }
    uint64_t bd = ~0ull;
    uint32_t bl = 0xFFFFFFFFu;
    nn_scan_tile<C, B>(packed, W, H, g.tiles_x, best_t, q_packed, kc, bd, bl);
    for (int st = 0; st < g.n_supers; ++st) {
        const int tx0 = (st % g.supers_x) * kSuper, ty0 = (st / g.supers_x) * kSuper;
        const uint64_t lbs = box_distance<C, B>(rep, __ldg(&sup[st]), kc);
        const uint32_t first_s = (uint32_t)(ty0 * kLutTile) * (uint32_t)W + (uint32_t)(tx0 * kLutTile);
        if (!(lbs < bd || (lbs == bd && first_s < bl))) continue;
        for (int ty = ty0; ty < min(ty0 + kSuper, g.tiles_y); ++ty)
            for (int tx = tx0; tx < min(tx0 + kSuper, g.tiles_x); ++tx) {
                const int t = ty * g.tiles_x + tx;
                if (t == best_t) continue;
                const uint64_t lb = box_distance<C, B>(rep, __ldg(&bounds[t]), kc);
                const uint32_t first = (uint32_t)(ty * kLutTile) * (uint32_t)W + (uint32_t)(tx * kLutTile);
                if (lb < bd || (lb == bd && first < bl))
                    nn_scan_tile<C, B>(packed, W, H, g.tiles_x, t, q_packed, kc, bd, bl);
            }
    }
    return (bl % (uint32_t)W) | ((bl / (uint32_t)W) << 16);
}

// The bin representative of guide value v keyed on key_bits per channel
// (channels from kc on zero), packed like v: the query of a table entry.
template <int C, int B>
__device__ __forceinline__ uint32_t bin_representative(uint32_t v, int key_bits, int kc) {
    using F = GuideFmt<C, B>;
    const int z = B - key_bits;
    uint32_t q = 0;
#pragma unroll
    for (int c = 0; c < C; ++c)
        if (c < kc) q |= (((F::chan(v, c) >> z) << z) + (((1u << z) - 1u) >> 1)) << (c * B);
    return q;
}

}  // namespace sb

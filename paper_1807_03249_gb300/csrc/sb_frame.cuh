// Per-frame StyleBlit kernels: Algorithm 2 (ParallelStyleBlit) with the
// coordinate transfer and voting step of Section 3.2.  Templates only; the
// sb_frame_*.cu files instantiate them per guide format.
//
// One CTA owns a 64 x TH output tile (TH = 32; the batch kernels also take
// 16 and 64).  The fused kernel computes the assignment A of the tile plus a
// halo of R pixels (the vote window) in shared memory, so A never reaches
// device memory:
//
//   phase 0  the seed cells of every level >= 3 (thread k builds cell k;
//            level 2 has many cells and is built only if a pixel of the tile
//            still needs it; level 1 has no cell table, its few pixels search
//            their seeds one by one).  A cell is: jitter hash -> seed q
//            clamped into the target -> G_T[q] -> table entry u*(q).  Cells
//            are stored column-major (x outer, y inner), each as (-2q, |q|^2)
//            in region-centred coordinates pre-scaled by 2^11 with the cell's
//            column-major index in the low 11 bits, plus the translation
//            u* - q packed.  Then the target guide of the region -> smem (one
//            packed uint32 per pixel, a warp per region row).
//   levels   for l = L..1 while pixels are pending: a pixel p takes the
//            minimum over its 3 x 3 cells of |q|^2 - 2 q.p (which orders seeds
//            like |q - p|^2) packed with the cell index: one min gives the
//            nearest seed and, on ties, the first cell in x-outer, y-inner
//            order, as NearestSeed's strict < does.  The candidate
//            s = u* + (p - q) is accepted if it lies in the source and
//            |G_S[s] - G_T[p]|^2 <= t (level 1 always accepts, s clamped).
//            Work goes by vertical segments of 4 pixels, one region column per
//            lane: a segment lies in one cell at levels >= 2 and the keys are
//            affine in p, so its four keys per cell are one multiply-add and
//            three adds.  Each warp compacts the segments it rejected into a
//            list of its own and takes them down the levels by itself.  The
//            level lists and, later, the vote's two pixel lists share one
//            area, and level 1 keeps no cells, so four CTAs leave most of the
//            SM's unified L1 / shared memory to the L1 cache.
//   vote     once A is complete, the region's assignments become style texel
//            indices (over the dead target guide) and ballots mark, per region
//            row, where A steps by exactly one pixel (E, horizontally), where
//            it continues the row above (V) and which assignments lie at least
//            R pixels inside the source (N).  One thread per region row turns
//            them into 64-bit masks of the output columns whose window row is
//            one run, at most two runs, or interior (over the dead seed
//            cells); four threads per output row AND them over the window and
//            list the row's pixels by class.  A window made of one translation
//            votes exactly C_S[A(p)], a plain copy; an interior window whose
//            rows have at most two runs sums one gather per run with no source
//            test; the rest (junctions, frame and source borders) sum tap by
//            tap.  Integer sums, round-half-up division.
//   store    uniform windows store from the copy pass (coalesced rows), the
//            others from the two list passes.
#pragma once

#include <atomic>
#include <climits>

#include "sb_internal.cuh"
#include "sb_nn.cuh"

namespace sb {

constexpr int kTW = 64;
constexpr int kTH = 32;        // default tile height (sb_stylize, sb_blend, sb_assign_chunks)

// A tile of 64 x TH output pixels: 8 * TH threads, four output rows per warp.
// Batches may use TH = 16, 32 or 64 (the autotuner's tile shapes).
template <int TH>
struct Tile {
    static_assert(TH == 16 || TH == 32 || TH == 64, "tile height");
    static constexpr int H = TH;
    static constexpr int Threads = 8 * TH;
    static constexpr int Warps = Threads / 32;
};
constexpr int kEagerMinLevel = 3;           // levels >= this get their cells in phase 0
constexpr int kKeyShift = 11;               // cell-index bits of the packed seed key
constexpr int kPackedMaxLevel = 8;          // levels whose packed keys fit 32 bits
// Packed-level cells hold u* - q (q region-centred) with this bias on both
// axes, packed x | y << 16: seeds of those levels lie within 600 pixels of the
// region centre, so both fields stay within 16 bits.
constexpr int kShiftBias = 1024;

enum Mode { kAssign = 0, kStylize = 1 };

struct FrameArgs {
    const uint8_t *tgt;
    int64_t tgt_stride;
    int W, H;
    const uint32_t *src_packed;  // G_S, one packed uint32 per pixel, row-major
    int Ws, Hs;
    const uint32_t *lut;         // table, or nullptr: query the search index
    const uint4 *nn_bounds;      // search index (keys wider than 24 bits)
    int key_bits;
    int key_channels;
    const uint8_t *style;
    int style_stride_px;         // style row stride in pixels (height * stride < 2^31)
    int levels;
    uint64_t threshold;
    uint32_t seed;
    int radius;
    const uint32_t *assign_in;   // sb_blend
    uint32_t *assign_out;        // sb_assign_chunks
    uint8_t *level_out;          // sb_assign_chunks (nullable)
    uint32_t *rgba_out;          // RGBA8 as one uint32 per pixel
    float4 *f32_out;             // sb_blend float variant
};

// upper bound of the cells of level l touching a region of RW x RH pixels
__host__ __device__ constexpr int cells_bound(int RW, int RH, int l) {
    return (((RW - 1) >> l) + 4) * (((RH - 1) >> l) + 4);
}

struct SmemLayout {
    int RW, RH, NR, NC;
    size_t off_cells, off_gt, off_A, off_lists, off_bytes, off_masks, off_cnt, total;
};

// Rows above the tile where the first segment (4 rows, starting at a target row
// that is a multiple of 4) starts: the blend radius rounded up to 4.
__host__ __device__ constexpr int seg_pad(int r) { return (r + 3) / 4 * 4; }

// Entries of one warp's pending-segment list: the most segments a warp takes
// at the top level (segments of 4 rows cover the region and the seg_pad rows
// above and below the tile).
__host__ __device__ constexpr int warp_list_cap(int r, int th) {
    return ((kTW + 2 * r) * ((th + 2 * seg_pad(r)) / 4) + 8 * th - 1) / (8 * th) * 32;
}

// Entries of the list area: during the assignment, two pending lists per
// warp (this level's and the next one's); during the vote, the tile's two
// pixel lists, whose classes are disjoint, one from each end.
__host__ __device__ constexpr int list_entries(int r, int th) {
    return 2 * (th / 4) * warp_list_cap(r, th) > th * kTW ? 2 * (th / 4) * warp_list_cap(r, th)
                                                           : th * kTW;
}

// Bytes of the vote's masks: per region row E, V, N (4 words each) and the
// 64-bit output-column masks hu, t2, vc, ni; per output row U, T2, NI.
__host__ __device__ constexpr size_t vote_mask_bytes(int r, int th) {
    return (size_t)(3 * 4 * 4 + 4 * 8) * (th + 2 * r) + (size_t)3 * 8 * th;
}

// Shared memory of one tile.  Once the assignment is done the seed cells and
// the region's target guide are dead: the vote lays its masks over the cells
// (the area is at least as large as the masks) and the source texel index of
// each region pixel's assignment over the guide.  The level bytes exist only
// for the assignment-only kernel (the fused path never stores levels).  Cells
// are kept for levels 2 and up (level 1 searches its seeds pixel by pixel), and
// one list area serves both the level loop and the vote.  The smaller the four
// CTAs' shared memory, the more of the SM's unified L1 / shared-memory array
// is left to the L1 cache that serves the exemplar gathers.
__host__ __device__ inline SmemLayout smem_layout(int r, int levels, bool level_bytes = false,
                                                  int th = kTH) {
    SmemLayout s;
    s.RW = kTW + 2 * r;
    s.RH = th + 2 * r;
    s.NR = s.RW * s.RH;
    s.NC = 0;
    for (int l = 2; l <= levels; ++l) s.NC += cells_bound(s.RW, s.RH, l);
    size_t o = 0;
    s.off_cells = o;
    s.off_masks = o;
    const size_t cell_bytes = sizeof(int4) * (size_t)s.NC, mask_bytes = vote_mask_bytes(r, th);
    o += (cell_bytes > mask_bytes ? cell_bytes : ((mask_bytes + 15) & ~(size_t)15));
    s.off_gt = o;
    o += sizeof(uint32_t) * (size_t)s.NR;
    s.off_A = o;
    o += sizeof(uint32_t) * (size_t)s.NR;
    s.off_lists = o;
    o += sizeof(uint16_t) * (size_t)list_entries(r, th);
    s.off_bytes = o;
    if (level_bytes) o += (size_t)s.NR;
    o = (o + 15) & ~(size_t)15;
    s.off_cnt = o;
    o += 32;  // 3 level counters (rotating), the vote's two list lengths
    s.total = o;
    return s;
}

// Seed cells of level l for the clamped region [xa, xb] x [ya, yb].
struct LevelCells {
    int cx0, cy0, ncx, ncy;
};

__device__ __forceinline__ LevelCells level_cells(int l, int xa, int xb, int ya, int yb) {
    LevelCells g;
    g.cx0 = (xa >> l) - 1;
    g.ncx = (xb >> l) - (xa >> l) + 3;
    g.cy0 = (ya >> l) - 1;
    g.ncy = (yb >> l) - (ya >> l) + 3;
    return g;
}

// Number of cells of levels l_hi down to l_lo for the clamped region.
__device__ __forceinline__ int cell_count(int l_hi, int l_lo, int xa, int xb, int ya, int yb) {
    int total = 0;
    for (int l = l_hi; l >= l_lo; --l) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        total += g.ncx * g.ncy;
    }
    return total;
}

// Cell k of the levels stacked from l_hi downwards (each column-major): its
// level, column-major index within the level and seed q (clamped into the
// target).
struct CellTask {
    int l, ci, sx, sy;
};

// Cell ci (column-major) of level l, whose cells are g.
__device__ __forceinline__ CellTask cell_at(const FrameArgs &a, int l, int ci,
                                            const LevelCells &g) {
    CellTask t;
    // column-major: ci = lcx * ncy + lcy
    // ci / ncy through a float reciprocal: ci < 2^11 and ncy < 2^6 keep the
    // true quotient at least 0.5 / ncy from an integer, far above the
    // rounding error, so the truncation is exact
    const int lcx = (int)(((float)ci + 0.5f) * __frcp_rn((float)g.ncy));
    const int lcy = ci - lcx * g.ncy;
    const int h = 1 << l;
    const int bx = g.cx0 + lcx, by = g.cy0 + lcy;
    const uint32_t hsh = cell_hash(level_key(a.seed, l), bx, by);
    const int ox = (int)(((hsh & 0xFFFFu) * (uint32_t)h) >> 16);
    const int oy = (int)(((hsh >> 16) * (uint32_t)h) >> 16);
    t.l = l;
    t.ci = ci;
    t.sx = min(max(bx * h + ox, 0), a.W - 1);
    t.sy = min(max(by * h + oy, 0), a.H - 1);
    return t;
}

__device__ __forceinline__ CellTask cell_task(const FrameArgs &a, int k, int l_hi, int xa, int xb,
                                              int ya, int yb) {
    int l = l_hi, off = 0;
    LevelCells g = level_cells(l, xa, xb, ya, yb);
    while (k >= off + g.ncx * g.ncy) {
        off += g.ncx * g.ncy;
        --l;
        g = level_cells(l, xa, xb, ya, yb);
    }
    return cell_at(a, l, k - off, g);
}

// The stored cell, in region-centred coordinates (q - (cxo, cyo)): levels
// with packed keys hold (-2q, |q|^2) scaled by 2^11 with the cell index added
// to |q|^2 (computed modulo 2^32: only the keys built from it, which fit 32
// bits, are used) and the translation u* - q biased by kShiftBias, packed, so
// a pixel's candidate u* + (p - q) is one add; coarser levels hold (-q, 0, u*)
// and their keys are squared distances in 64 bits.
__device__ __forceinline__ int4 cell_value(const CellTask &t, uint32_t u, int cxo, int cyo) {
    const int qx = t.sx - cxo, qy = t.sy - cyo;
    if (t.l <= kPackedMaxLevel) {
        constexpr uint32_t S = 1u << kKeyShift;
        const uint32_t z = ((uint32_t)(qx * qx) + (uint32_t)(qy * qy)) * S + (uint32_t)t.ci;
        const uint32_t d = (uint32_t)((int)(u & 0xFFFFu) - qx + kShiftBias) |
                           ((uint32_t)((int)(u >> 16) - qy + kShiftBias) << 16);
        return make_int4((int)((uint32_t)(-2 * qx) * S), (int)((uint32_t)(-2 * qy) * S), (int)z,
                         (int)d);
    }
    return make_int4(-qx, -qy, 0, (int)u);
}

// Packed region-centred position (px, py) minus the bias: added to a cell's
// packed translation it gives the packed candidate.  A coordinate below zero
// borrows and lands far above any source side (in_source fails).
__device__ __forceinline__ uint32_t biased_pos(int px, int py) {
    return (uint32_t)((px - kShiftBias) + (py - kShiftBias) * 65536);
}

// u*(q) of a seed whose target guide value is g (Algorithm 2, "found via
// lookup"): the table entry of g's bin, or, for keys wider than a table, the
// search index queried at the bin representative (the same source position).
template <int C, int B>
__device__ __forceinline__ uint32_t seed_source(const FrameArgs &a, uint32_t g) {
    using F = GuideFmt<C, B>;
    if (a.lut) return __ldg(a.lut + F::key(g, a.key_bits, a.key_channels));
    return nn_query<C, B>(a.src_packed, a.nn_bounds, a.Ws, a.Hs,
                          bin_representative<C, B>(g, a.key_bits, a.key_channels), a.key_channels);
}

// Builds cells k0, k0 + NT, ... (NT threads) of the levels l_hi down to l_lo into
// cells[base_hi + k].
template <int C, int B, int NT>
__device__ __forceinline__ void build_cells(const FrameArgs &a, int4 *cells, int l_hi, int l_lo,
                                            int base_hi, int xa, int xb, int ya, int yb,
                                            int cxo, int cyo, int k0 = 0, int total = -1) {
    using F = GuideFmt<C, B>;
    if (total < 0) total = cell_count(l_hi, l_lo, xa, xb, ya, yb);
#pragma unroll 1
    for (int k = k0 + (int)threadIdx.x; k < total; k += NT) {
        const CellTask t = cell_task(a, k, l_hi, xa, xb, ya, yb);
        const uint32_t u = seed_source<C, B>(a, F::load(a.tgt, a.tgt_stride, t.sx, t.sy));
        cells[base_hi + k] = cell_value(t, u, cxo, cyo);
    }
}

// Vertical segments of 4 pixels starting at target rows that are multiples of
// 4 cover the region (the tile plus its R halo): segment s takes region column
// s % RW, so the lanes of a warp hold neighbouring columns.  At every level
// >= 2 a segment lies inside one seed cell.
template <int R, int TH>
struct Segs {
    static constexpr int kPad = seg_pad(R);  // first segment row: kPad rows above the tile
    static constexpr int RW = kTW + 2 * R, RH = TH + 2 * R;
    static constexpr int NSY = (TH + 2 * kPad) / 4;
    static constexpr int NS = RW * NSY;
    __device__ __forceinline__ static int rx(int s) { return s % RW; }
    __device__ __forceinline__ static int ry(int s) { return 4 * (s / RW) - kPad + R; }
    // bit j: lo <= ry + j < hi
    __device__ __forceinline__ static uint32_t span(int ry, int lo, int hi) {
        const int a = min(max(lo - ry, 0), 4), b = min(max(hi - ry, 0), 4);
        return ((1u << b) - 1u) & ~((1u << a) - 1u);
    }
    // bit j: row ry + j lies in the region
    __device__ __forceinline__ static uint32_t rows(int ry) { return span(ry, 0, RH); }
};

// The region's columns [c_lo, c_hi) and rows [r_lo, r_hi) inside the target.
struct TileBounds {
    int c_lo, c_hi, r_lo, r_hi;
    template <int R, int TH>
    __device__ __forceinline__ static TileBounds of(int rx0, int ry0, int W, int H) {
        return TileBounds{max(0, -rx0), min(kTW + 2 * R, W - rx0), max(0, -ry0),
                          min(TH + 2 * R, H - ry0)};
    }
    // bit j: pixel (rx, ry + j) of a segment lies in the region and the target
    template <int R, int TH>
    __device__ __forceinline__ uint32_t mask(int rx, int ry) const {
        return rx >= c_lo && rx < c_hi ? Segs<R, TH>::span(ry, r_lo, r_hi) : 0u;
    }
};

// The source side of a candidate test.
struct SrcView {
    const uint32_t *src_packed;
    int Ws, Hs;
    uint64_t threshold;
    // packed position v = x | y << 16 inside the source
    __device__ __forceinline__ bool in_source(uint32_t v) const {
        return (v & 0xFFFFu) < (uint32_t)Ws && v < ((uint32_t)Hs << 16);
    }
};

// Candidate test of the pixels of one segment: pixel j sits at region index
// ibase + j * RW and its candidate source position is the packed v[j].
// Accepted pixels get A (and the level); the bits of rejected pixels of m
// are returned.
template <int C, int B, int RW>
__device__ __forceinline__ uint32_t test_segment(const SrcView &a, const uint32_t *gt,
                                                 uint32_t *A, uint8_t *lev, int l, uint32_t t32,
                                                 uint32_t m, int ibase, const uint32_t (&v)[4]) {
    using F = GuideFmt<C, B>;
    uint32_t gsv[4];
    bool ok[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ok[j] = ((m >> j) & 1u) && a.in_source(v[j]);
        gsv[j] = ok[j] ? __ldg(a.src_packed + ((v[j] >> 16) * (uint32_t)a.Ws + (v[j] & 0xFFFFu)))
                       : 0u;
    }
    uint32_t rej = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!((m >> j) & 1u)) continue;
        bool acc = false;
        if (ok[j]) {
            const uint64_t d = F::dist(gsv[j], gt[ibase + j * RW]);
            if constexpr (B == 8) acc = (uint32_t)d <= t32;
            else acc = d <= a.threshold;
        }
        if (acc) {
            A[ibase + j * RW] = v[j];
            if (lev) lev[ibase + j * RW] = (uint8_t)l;
        }
        rej |= (uint32_t)!acc << j;
    }
    return rej;
}

// Level 1 (seed spacing 2; a segment spans two cells), pixel by pixel and
// without a cell table: each pixel hashes its own 3 x 3 seed cells, keeps the
// nearest seed in NearestSeed's order (x outer, y inner, first minimum), looks
// the seed's guide up (table or search index) and takes the candidate clamped
// into the source: the finest level accepts every pixel.  Few pixels reach
// level 1, so a table of the region's level-1 cells would cost more shared
// memory than building it saves.  It runs in a pass of its own after the
// other levels (its state stays out of the registers of their loops).
template <int C, int B, int R, int TH>
__device__ __forceinline__ void segment_level1(const FrameArgs &a, uint32_t *A, uint8_t *lev,
                                               int rx0, int ry0, int rx, int ry, uint32_t m) {
    using F = GuideFmt<C, B>;
    constexpr int RW = Segs<R, TH>::RW;
    const uint32_t lk = level_key(a.seed, 1);
    const int px = rx0 + rx;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        if (!((m >> j) & 1u)) continue;
        const int py = ry0 + ry + j;
        int best = INT_MAX, qx = 0, qy = 0;
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            const int bx = (px >> 1) + d / 3 - 1, by = (py >> 1) + d % 3 - 1;
            const uint32_t h = cell_hash(lk, bx, by);
            // offsets floor(2 j) of the 16-bit jitter fractions
            const int sx = min(max(2 * bx + (int)((h & 0xFFFFu) >> 15), 0), a.W - 1);
            const int sy = min(max(2 * by + (int)(h >> 31), 0), a.H - 1);
            const int dist = (sx - px) * (sx - px) + (sy - py) * (sy - py);
            if (dist < best) {
                best = dist;
                qx = sx;
                qy = sy;
            }
        }
        const uint32_t u = seed_source<C, B>(a, F::load(a.tgt, a.tgt_stride, qx, qy));
        const int sx = min(max((int)(u & 0xFFFFu) + px - qx, 0), a.Ws - 1);
        const int sy = min(max((int)(u >> 16) + py - qy, 0), a.Hs - 1);
        const int i = (ry + j) * RW + rx;
        A[i] = (uint32_t)sx | ((uint32_t)sy << 16);
        if (lev) lev[i] = 1;
    }
}

// Levels above kPackedMaxLevel, where every pixel searches its own seed (keys
// are 64-bit squared distances packed with the cell index).  They are rare,
// so pixels go one at a time with little live state (the common path keeps
// its registers).
template <int C, int B, int R, int TH>
__device__ __forceinline__ uint32_t segment_level_rare(const SrcView &a, const uint32_t *gt,
                                                       uint32_t *A, uint8_t *lev,
                                                       const int4 *cells, int base, int c0,
                                                       int ncy, int l, uint32_t t32, int rx,
                                                       int ry, uint32_t m) {
    using F = GuideFmt<C, B>;
    constexpr int RW = Segs<R, TH>::RW, RH = Segs<R, TH>::RH;
    constexpr int kMask = (1 << kKeyShift) - 1;
    const int prx = rx - RW / 2, pry = ry - RH / 2;
    uint32_t rej = 0;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        if (!((m >> j) & 1u)) continue;
        long long key = LLONG_MAX;
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            const int c = c0 + (d / 3 - 1) * ncy + (d % 3 - 1);
            const int4 cl = cells[c];
            const long long dx = prx + cl.x, dy = pry + j + cl.y;
            key = min(key, ((dx * dx + dy * dy) << kKeyShift) | (c - base));
        }
        // these cells hold u* and -q
        const int4 cl = cells[base + (int)(key & kMask)];
        const int sx = (int)((uint32_t)cl.w & 0xFFFFu) + prx + cl.x;
        const int sy = (int)((uint32_t)cl.w >> 16) + pry + j + cl.y;
        const int i = (ry + j) * RW + rx;
        bool acc = (unsigned)sx < (unsigned)a.Ws && (unsigned)sy < (unsigned)a.Hs;
        if (acc) {
            const uint64_t d = F::dist(
                __ldg(a.src_packed + ((uint32_t)sy * (uint32_t)a.Ws + (uint32_t)sx)), gt[i]);
            if constexpr (B == 8) acc = (uint32_t)d <= t32;
            else acc = d <= a.threshold;
        }
        if (acc) {
            A[i] = (uint32_t)sx | ((uint32_t)sy << 16);
            if (lev) lev[i] = (uint8_t)l;
        } else {
            rej |= 1u << j;
        }
    }
    return rej;
}

// Level l (2 <= l <= kMaxLevels) of the pixels m of the segment at
// region (rx, ry): returns the rejected ones.  The packed keys of the nine
// candidates are affine in p, so the pixels that pick a given seed form a
// convex set: when the first and last pixel of m pick the same seed, every
// pixel between them does and the nine-way search runs once.  Otherwise each
// pixel searches (the unscaled levels: segment_level_rare).
template <int C, int B, int R, int TH>
__device__ __forceinline__ uint32_t segment_level(const FrameArgs &a, const uint32_t *gt,
                                                  uint32_t *A, uint8_t *lev, const int4 *cells,
                                                  int base, const LevelCells &g, int l, int rx0,
                                                  int ry0, uint32_t t32, int rx, int ry,
                                                  uint32_t m) {
    using S = Segs<R, TH>;
    constexpr int RW = S::RW, RH = S::RH;
    constexpr int kMask = (1 << kKeyShift) - 1;
    const int prx = rx - RW / 2, pry = ry - RH / 2;
    const int c0 = base + (((rx0 + rx) >> l) - g.cx0) * g.ncy + (((ry0 + ry) >> l) - g.cy0);
    const int ibase = ry * RW + rx;
    const SrcView sv{a.src_packed, a.Ws, a.Hs, a.threshold};
    if (l > kPackedMaxLevel)
        return segment_level_rare<C, B, R, TH>(sv, gt, A, lev, cells, base, c0, g.ncy, l, t32, rx, ry,
                                           m);
    // every lane evaluates the nine keys at all four pixels (three adds per
    // cell on top of the first pixel's key): no lane waits for a neighbour
    // whose segment straddles a Voronoi edge
    int k[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
#pragma unroll 1
    for (int dx = -1; dx <= 1; ++dx) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int4 cl = cells[c0 + dx * g.ncy + dy];
            // modulo 2^32: the keys themselves fit 32 bits
            uint32_t e = (uint32_t)cl.z + (uint32_t)cl.x * (uint32_t)prx +
                         (uint32_t)cl.y * (uint32_t)pry;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                k[j] = min(k[j], (int)e);
                e += (uint32_t)cl.y;
            }
        }
    }
    // candidate of pixel j: its seed cell's packed translation plus p
    const uint32_t P = biased_pos(prx, pry);
    uint32_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = (uint32_t)cells[base + (k[j] & kMask)].w + P + (j << 16);
    return test_segment<C, B, RW>(sv, gt, A, lev, l, t32, m, ibase, v);
}

// ---------------------------------------------------------------------------
// assignment of the region held in shared memory (Algorithm 2)
// ---------------------------------------------------------------------------
template <int C, int B, int R, int TH>
__device__ __forceinline__ void assign_region(const FrameArgs &a, const SmemLayout &L, int rx0,
                                              int ry0, unsigned char *smem, uint8_t *lev) {
    using F = GuideFmt<C, B>;
    constexpr int RW = kTW + 2 * R, RH = TH + 2 * R;
    constexpr int kThreads = Tile<TH>::Threads;
    int4 *cells = reinterpret_cast<int4 *>(smem + L.off_cells);
    uint32_t *gt = reinterpret_cast<uint32_t *>(smem + L.off_gt);
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
    uint16_t *const lists = reinterpret_cast<uint16_t *>(smem + L.off_lists);
    const int tid = threadIdx.x;

    const int xa = max(rx0, 0), xb = min(rx0 + RW, a.W) - 1;
    const int ya = max(ry0, 0), yb = min(ry0 + RH, a.H) - 1;
    const int cxo = rx0 + RW / 2, cyo = ry0 + RH / 2;
    const uint32_t t32 = a.threshold > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)a.threshold;
    const int L_top = a.levels;
    // levels with a cell table: L_top down to 2 (level 1 has none)
    const int eager_lo = L_top <= kEagerMinLevel ? 2 : kEagerMinLevel;
    const TileBounds tb = TileBounds::of<R, TH>(rx0, ry0, a.W, a.H);

    // phase 0: thread k builds eager cell k (levels L_top .. eager_lo
    // stacked, each column-major; the level of its cell is found while
    // counting them), then every load of the region's guide is issued before
    // the first store that waits on one.  Finishing the cell first keeps its
    // state out of the registers that hold the guide loads.
    int n_eager = 0, my_l = 0, my_ci = 0;
    LevelCells my_g{};
    for (int l = L_top; l >= eager_lo; --l) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        const int n = g.ncx * g.ncy;
        if (tid >= n_eager && tid < n_eager + n) {
            my_l = l;
            my_ci = tid - n_eager;
            my_g = g;
        }
        n_eager += n;
    }
    const bool has_cell = tid < n_eager;
    if (has_cell) {
        const CellTask ct = cell_at(a, my_l, my_ci, my_g);
        const uint32_t cu = seed_source<C, B>(a, F::load(a.tgt, a.tgt_stride, ct.sx, ct.sy));
        cells[tid] = cell_value(ct, cu, cxo, cyo);
    }
    // the region's guide: a warp per region row for columns 0..63 (lanes x
    // and 32 + x; one row address per lane and row), and the last 2R columns
    // of 32 / 2R rows at once (lane = row * 2R + column); every load is
    // issued before the first store
    constexpr int kWarps = Tile<TH>::Warps;
    constexpr int kRowIt = (RH + kWarps - 1) / kWarps;
    constexpr int kCw = R > 0 ? 2 * R : 1, kTRows = 32 / kCw;
    constexpr int kTailIt = R > 0 ? ((RH + kTRows - 1) / kTRows + kWarps - 1) / kWarps : 0;
    static_assert(2 * kRowIt + kTailIt <= 32, "inside bits");
    const int wp = tid >> 5, ln = tid & 31;
    const int t_rl = ln / kCw, t_col = ln - t_rl * kCw;
    uint32_t gv[kRowIt][2], gw[kTailIt > 0 ? kTailIt : 1];
    uint32_t inside = 0;  // bit 2j + c: main pixel (j, c); bit 2 kRowIt + j: tail pixel j
    {
        // row address stepped by kWarps rows (only dereferenced inside the target)
        const uint8_t *row = a.tgt + (int64_t)(ry0 + wp) * a.tgt_stride;
        const int64_t step = (int64_t)kWarps * a.tgt_stride;
#pragma unroll
        for (int j = 0; j < kRowIt; ++j) {
            const int ry = wp + j * kWarps, gy = ry0 + ry;
            const bool rowin = (j + 1 < kRowIt || ry < RH) && (unsigned)gy < (unsigned)a.H;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int gx = rx0 + c * 32 + ln;
                const bool in = rowin && (unsigned)gx < (unsigned)a.W;
                gv[j][c] = in ? F::load(row, 0, gx, 0) : 0u;
                inside |= (uint32_t)in << (2 * j + c);
            }
            row += step;
        }
    }
#pragma unroll
    for (int j = 0; j < kTailIt; ++j) {
        const int ry = (wp + j * kWarps) * kTRows + t_rl;
        const int gx = rx0 + kTW + t_col, gy = ry0 + ry;
        const bool in = t_rl < kTRows && ry < RH && (unsigned)gx < (unsigned)a.W &&
                        (unsigned)gy < (unsigned)a.H;
        gw[j] = in ? F::load(a.tgt, a.tgt_stride, gx, gy) : 0u;
        inside |= (uint32_t)in << (2 * kRowIt + j);
    }
#pragma unroll
    for (int j = 0; j < kRowIt; ++j) {
        const int ry = wp + j * kWarps;
        if (j + 1 < kRowIt || ry < RH) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int i = ry * RW + c * 32 + ln;
                if ((inside >> (2 * j + c)) & 1u) gt[i] = gv[j][c];
                else A[i] = kInvalid;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kTailIt; ++j) {
        const int ry = (wp + j * kWarps) * kTRows + t_rl;
        if (t_rl < kTRows && ry < RH) {
            const int i = ry * RW + kTW + t_col;
            if ((inside >> (2 * kRowIt + j)) & 1u) gt[i] = gw[j];
            else A[i] = kInvalid;
        }
    }
    if (n_eager > kThreads)
        build_cells<C, B, kThreads>(a, cells, L_top, eager_lo, 0, xa, xb, ya, yb, cxo, cyo, kThreads,
                                    n_eager);
    __syncthreads();

    // The top level visits every segment of the region, thread by thread as
    // the block's segments fall (warp w takes 32 consecutive segments of each
    // round); every warp keeps the segments it rejected (entries: segment
    // index << 4 | pixel mask) in a list of its own and takes them down the
    // eager levels by itself, compacting with ballots: no block barrier and no
    // shared counter between those levels.  Level 2 needs its cells built by
    // the whole block first, and only if some warp still holds a pixel; level
    // 1 goes pixel by pixel without cells.
    using S = Segs<R, TH>;
    constexpr int kWarpCap = warp_list_cap(R, TH);
    static_assert(kWarpCap == (S::NS + kThreads - 1) / kThreads * 32, "list capacity");
    const int warp = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint16_t *wl_cur = lists + warp * kWarpCap, *wl_nxt = lists + (kWarps + warp) * kWarpCap;
    int n_w = 0, base = 0;
    {
        const LevelCells g = level_cells(L_top, xa, xb, ya, yb);
        for (int s0 = 0; s0 < S::NS; s0 += kThreads) {
            const int sg = s0 + tid;
            const uint32_t m = sg < S::NS ? tb.template mask<R, TH>(S::rx(sg), S::ry(sg)) : 0u;
            // a hierarchy of one level leaves every pixel to the level-1 pass
            uint32_t rej = L_top == 1 ? m : 0u;
            if (m && L_top > 1)
                rej = segment_level<C, B, R, TH>(a, gt, A, lev, cells, base, g, L_top, rx0, ry0,
                                                 t32, S::rx(sg), S::ry(sg), m);
            const unsigned mk = __ballot_sync(0xFFFFFFFFu, rej != 0);
            if (rej) wl_cur[n_w + __popc(mk & lt)] = (uint16_t)((sg << 4) | (int)rej);
            n_w += __popc(mk);
        }
        base += g.ncx * g.ncy;
    }
    bool synced = false;  // block-uniform
    for (int l = L_top - 1; l >= 2; --l) {
        if (l == kEagerMinLevel - 1 && eager_lo > 2) {
            // level 2: the block builds its cells, and only if some warp
            // still holds a pixel (every thread reaches this point; when none
            // does, this barrier is also the one that completes A)
            if (!__syncthreads_or(n_w > 0)) {
                synced = true;
                break;
            }
            build_cells<C, B, kThreads>(a, cells, 2, 2, base, xa, xb, ya, yb, cxo, cyo);
            __syncthreads();
        }
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        // n_w is the same in every lane of the warp
        int n_next = 0;
        for (int j0 = 0; j0 < n_w; j0 += 32) {
            const uint32_t e = j0 + lane < n_w ? wl_cur[j0 + lane] : 0u;
            const uint32_t m = e & 15u;
            const int sg = (int)(e >> 4);
            uint32_t rej = 0;
            if (m)
                rej = segment_level<C, B, R, TH>(a, gt, A, lev, cells, base, g, l, rx0, ry0, t32,
                                                 S::rx(sg), S::ry(sg), m);
            const unsigned mk = __ballot_sync(0xFFFFFFFFu, rej != 0);
            if (rej) wl_nxt[n_next + __popc(mk & lt)] = (uint16_t)((sg << 4) | (int)rej);
            n_next += __popc(mk);
        }
        __syncwarp();
        uint16_t *const t = wl_cur;
        wl_cur = wl_nxt;
        wl_nxt = t;
        n_w = n_next;
        base += g.ncx * g.ncy;
    }
    // level 1: the pixels still pending, each warp its own list
    for (int j0 = 0; j0 < n_w; j0 += 32) {
        const uint32_t e = j0 + lane < n_w ? wl_cur[j0 + lane] : 0u;
        const int sg = (int)(e >> 4);
        if (e & 15u) segment_level1<C, B, R, TH>(a, A, lev, rx0, ry0, S::rx(sg), S::ry(sg), e & 15u);
    }
    if (!synced) __syncthreads();  // the region's A is complete before the vote reads it
}

// ---------------------------------------------------------------------------
// voting over the tile (Section 3.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 rgba_f32(uint32_t col) {
    return make_float4(__fdiv_rn((float)(col & 0xFF), 255.f),
                       __fdiv_rn((float)((col >> 8) & 0xFF), 255.f),
                       __fdiv_rn((float)((col >> 16) & 0xFF), 255.f),
                       __fdiv_rn((float)(col >> 24), 255.f));
}

// Channel sums of a vote.  Windows of at most 15 x 15 taps keep two channels
// per 32-bit word (16-bit lanes: 225 * 255 < 2^16); larger ones one per word.
template <bool kPacked>
struct VoteAcc;

template <>
struct VoteAcc<true> {
    uint32_t lo = 0, hi = 0, n = 0;  // lo = c0 | c2 << 16, hi = c1 | c3 << 16
    __device__ __forceinline__ void add(uint32_t col, uint32_t cnt) {
        sum(col, cnt);
        n += cnt;
    }
    // cnt taps of colour col, the count kept by the caller
    __device__ __forceinline__ void sum(uint32_t col, uint32_t cnt) {
        lo += (col & 0x00FF00FFu) * cnt;
        hi += __byte_perm(col, 0u, 0x4341u) * cnt;  // bytes 1 and 3 into the low halves
    }
    __device__ __forceinline__ void sums(uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                         uint32_t &s3) const {
        s0 = lo & 0xFFFFu;
        s2 = lo >> 16;
        s1 = hi & 0xFFFFu;
        s3 = hi >> 16;
    }
};

template <>
struct VoteAcc<false> {
    uint32_t s[4] = {0, 0, 0, 0}, n = 0;
    __device__ __forceinline__ void add(uint32_t col, uint32_t cnt) {
        sum(col, cnt);
        n += cnt;
    }
    __device__ __forceinline__ void sum(uint32_t col, uint32_t cnt) {
        s[0] += (col & 0xFFu) * cnt;
        s[1] += ((col >> 8) & 0xFFu) * cnt;
        s[2] += ((col >> 16) & 0xFFu) * cnt;
        s[3] += (col >> 24) * cnt;
    }
    __device__ __forceinline__ void sums(uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                         uint32_t &s3) const {
        s0 = s[0];
        s1 = s[1];
        s2 = s[2];
        s3 = s[3];
    }
};

// Round-half-up quotient (s + n/2) / n for n >= 1 via a multiply-high:
// floor(y / n) == umulhi(y, floor((2^32 - 1) / n) + 1) for every n in
// [2, 961] and y <= 255 n + n / 2 (checked exhaustively); n == 1 is y.
__device__ __forceinline__ uint32_t div_round(uint32_t s, uint32_t n, uint32_t m) {
    const uint32_t y = s + (n >> 1);
    return n == 1 ? y : __umulhi(y, m);
}

template <bool F32, int R, typename Acc>
__device__ __forceinline__ void vote_store(const FrameArgs &a, const Acc &acc, int gx, int gy) {
    uint32_t s0, s1, s2, s3;
    acc.sums(s0, s1, s2, s3);
    const uint32_t n = acc.n;
    if constexpr (F32) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n) {
            const float dn = (float)(255u * n);
            o = make_float4(__fdiv_rn((float)s0, dn), __fdiv_rn((float)s1, dn),
                            __fdiv_rn((float)s2, dn), __fdiv_rn((float)s3, dn));
        }
        a.f32_out[(int64_t)gy * a.W + gx] = o;
    } else {
        uint32_t o = 0;
        if (n) {
            // a full window (the common case) divides by a constant
            constexpr uint32_t kFull = (2 * R + 1) * (2 * R + 1);
            const uint32_t m = n == kFull ? 0xFFFFFFFFu / kFull + 1u : 0xFFFFFFFFu / n + 1u;
            o = div_round(s0, n, m) | (div_round(s1, n, m) << 8) | (div_round(s2, n, m) << 16) |
                (div_round(s3, n, m) << 24);
        }
        a.rgba_out[(int64_t)gy * a.W + gx] = o;
    }
}

// Source position of window tap o = (ox, oy) of a neighbour whose assignment
// is An: v = A(p + o) - o, packed x | y << 16.  A coordinate that drops below
// zero borrows and lands far above any source side, so in_source() rejects
// it; so does every tap of a neighbour outside the target (kInvalid).
__device__ __forceinline__ uint32_t tap_pos(uint32_t An, int ox, int oy) {
    return An - (uint32_t)(ox + oy * 65536);
}

struct StyleView {
    const uint32_t *style32;
    uint32_t stride, Ws, Hs16;  // row stride in pixels, source width, source height << 16
    __device__ __forceinline__ static StyleView of(const FrameArgs &a) {
        return StyleView{reinterpret_cast<const uint32_t *>(a.style), (uint32_t)a.style_stride_px,
                         (uint32_t)a.Ws, (uint32_t)a.Hs << 16};
    }
    __device__ __forceinline__ bool in_source(uint32_t v) const {
        return (v & 0xFFFFu) < Ws && v < Hs16;
    }
    __device__ __forceinline__ uint32_t at(uint32_t v) const { return texel(lin(v)); }
    // texel index y * stride + x of the packed source position v = x | y << 16
    __device__ __forceinline__ uint32_t lin(uint32_t v) const {
        return (v >> 16) * stride + (v & 0xFFFFu);
    }
    __device__ __forceinline__ uint32_t texel(uint32_t i) const { return __ldg(style32 + i); }
    // cnt taps whose source position is v (nothing when cnt == 0 or v is
    // outside the source)
    template <typename Acc>
    __device__ __forceinline__ void add(Acc &acc, uint32_t v, uint32_t cnt) const {
        const bool ok = cnt != 0u && in_source(v);
        acc.add(ok ? at(v) : 0u, ok ? cnt : 0u);
    }
};

// Step bits of window row ry for output column tx: bit i (0 <= i < 2R) is set
// when taps i and i + 1 of that row belong to one run (A steps by exactly one
// pixel between them).  E holds four words per region row (the fourth zero).
template <int R>
__device__ __forceinline__ uint32_t window_steps(const uint32_t *E, int ry, int tx) {
    constexpr uint32_t kM = (1u << (2 * R)) - 1u;
    const uint32_t *e = E + ry * 4;
    const int b = tx + 1;
    return __funnelshift_r(e[b >> 5], e[(b >> 5) + 1], b & 31) & kM;
}

// Windows whose rows have at most two runs each and whose taps all come from
// interior assignments (every tap lies in the source, so the window counts
// all (2R + 1)^2 taps): one gather per run (the second has length 0 in a
// single-run row).  T holds the texel index of each region pixel's
// assignment; tap o = (ox, oy) of a window reads texel T(p + o) - ox - oy S.
template <int R, bool F32, int NT>
__device__ __forceinline__ void vote_two_runs(const FrameArgs &a, const StyleView &sv,
                                              const uint32_t *T, const uint32_t *E,
                                              const uint16_t *list, int n, int x0, int y0) {
    constexpr int RW = kTW + 2 * R;
    constexpr bool kPacked = (2 * R + 1) * (2 * R + 1) * 255 < 65536;
    constexpr uint32_t kFull = (2 * R + 1) * (2 * R + 1);
    const uint32_t S = sv.stride;
    for (int j = threadIdx.x; j < n; j += NT) {
        const int k = list[j];
        const int tx = k % kTW, ty = k / kTW;
        VoteAcc<kPacked> acc;
        uint32_t rb = (uint32_t)R + (uint32_t)R * S;  // R - oy S
        // windows above 15 x 15 (one CTA per SM, rarely used) stay rolled
        constexpr int kUnroll = R <= 7 ? 2 * R + 1 : 1;
#pragma unroll kUnroll
        for (int oy = -R; oy <= R; ++oy) {
            const int ry = ty + R + oy;
            const uint32_t *row = T + ry * RW + tx;
            const uint32_t j1 = __ffs(~window_steps<R>(E, ry, tx));  // first run: taps [0, j1)
            acc.sum(sv.texel(row[0] + rb), j1);
            const uint32_t d = min(j1, 2u * R);
            acc.sum(sv.texel(row[d] + rb - d), 2u * R + 1u - j1);
            rb -= S;
        }
        acc.n = kFull;
        vote_store<F32, R>(a, acc, x0 + tx, y0 + ty);
    }
}

// Every other window (junctions of three or more chunks, frame borders and
// taps near the source border): tap by tap.  The block's such pixels share
// one list, stored downwards from `list` (entry j at list[-j]); an entry's top
// bit marks a window whose taps all come from interior assignments, which
// skips the per-tap source test.
constexpr uint16_t kInteriorFlag = 0x8000u;

template <int R, bool F32, int NT>
__device__ __forceinline__ void vote_taps(const FrameArgs &a, const StyleView &sv,
                                          const uint32_t *A, const uint32_t *T,
                                          const uint16_t *list, int n, int x0, int y0) {
    constexpr int RW = kTW + 2 * R;
    constexpr bool kPacked = (2 * R + 1) * (2 * R + 1) * 255 < 65536;
    constexpr uint32_t kFull = (2 * R + 1) * (2 * R + 1);
    constexpr int kUnroll = R <= 7 ? 2 * R + 1 : 1;
    const uint32_t S = sv.stride;
    for (int j = threadIdx.x; j < n; j += NT) {
        const int e = list[-j];  // the list runs downwards
        const int k = e & ~(int)kInteriorFlag;
        const int tx = k % kTW, ty = k / kTW;
        VoteAcc<kPacked> acc;
        if (e & kInteriorFlag) {
            uint32_t rb = (uint32_t)R * S;  // -oy S
            for (int oy = -R; oy <= R; ++oy) {
                const uint32_t *row = T + (ty + R + oy) * RW + tx + R;
#pragma unroll kUnroll
                for (int ox = -R; ox <= R; ++ox) acc.sum(sv.texel(row[ox] + rb - (uint32_t)ox), 1u);
                rb -= S;
            }
            acc.n = kFull;
            vote_store<F32, R>(a, acc, x0 + tx, y0 + ty);
        } else {
            for (int oy = -R; oy <= R; ++oy) {
                const uint32_t *row = A + (ty + R + oy) * RW + tx + R;
#pragma unroll kUnroll
                for (int ox = -R; ox <= R; ++ox) sv.add(acc, tap_pos(row[ox], ox, oy), 1u);
            }
            vote_store<F32, R>(a, acc, x0 + tx, y0 + ty);
        }
    }
}

// bits [j, j + 64) of the 128-bit value hi:lo, 0 <= j < 64
__device__ __forceinline__ uint64_t shr128(uint64_t lo, uint64_t hi, int j) {
    return j == 0 ? lo : ((lo >> j) | (hi << (64 - j)));
}

// Shared-memory words of the vote's masks: per region row E, V, N (4 words
// each) and the 64-bit output-column masks hu, t2, vc, ni; per output row the
// 64-bit class masks U, T2, NI.
template <int R, int TH>
struct VoteMasks {
    static constexpr int RH = TH + 2 * R;
    uint32_t *E, *V, *N;
    uint64_t *hu, *t2, *vc, *ni, *U, *T2, *NI;
    __device__ __forceinline__ static VoteMasks at(unsigned char *p) {
        VoteMasks m;
        m.E = reinterpret_cast<uint32_t *>(p);
        m.V = m.E + 4 * RH;
        m.N = m.V + 4 * RH;
        m.hu = reinterpret_cast<uint64_t *>(m.N + 4 * RH);
        m.t2 = m.hu + RH;
        m.vc = m.t2 + RH;
        m.ni = m.vc + RH;
        m.U = m.ni + RH;
        m.T2 = m.U + TH;
        m.NI = m.T2 + TH;
        return m;
    }
};

// texel index of a region pixel without an assignment in the source
constexpr uint32_t kNoTexel = 0xFFFFFFFFu;

// Step, link and interior bits of region pixel x of row ry (x >= 1 or
// ry >= 1 may fail at the region's first column or row), and its texel index.
template <int R, int RW, bool kTrustA>
__device__ __forceinline__ void pixel_bits(const uint32_t *A, uint32_t *T, const StyleView &sv,
                                           uint32_t iw, uint32_t ih16, int ry, int x, bool &eb,
                                           bool &vb, bool &nb) {
    constexpr uint32_t kRR = (uint32_t)R | ((uint32_t)R << 16);
    const int i = ry * RW + x;
    const uint32_t cur = A[i];
    eb = x >= 1 && cur == A[i - 1] + 1u;
    vb = ry >= 1 && cur == A[i - RW] + 0x10000u;
    // x - R borrows from y when x < R, which leaves the low half at or above
    // 65536 - R > iw
    const uint32_t d = cur - kRR;
    nb = (d & 0xFFFFu) < iw && d < ih16;
    // the fused kernels assign every target pixel a source position and mark
    // the rest kInvalid; assignments read from memory may be anything
    const bool ok = kTrustA ? cur != kInvalid : sv.in_source(cur);
    T[i] = ok ? sv.lin(cur) : kNoTexel;
}

// Exclusive prefix over the warp of v, and the warp's total in *tot.
__device__ __forceinline__ int warp_exclusive_scan(int v, int &tot) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    tot = __shfl_sync(0xFFFFFFFFu, x, 31);
    return x - v;
}

template <int R, bool F32, int TH, bool kTrustA = true>
__device__ __forceinline__ void vote_tile(const FrameArgs &a, const SmemLayout &L, int x0,
                                          int y0, const uint32_t *A, unsigned char *smem) {
    constexpr int RW = kTW + 2 * R, RH = TH + 2 * R;
    constexpr int kThreads = Tile<TH>::Threads, kWarps = Tile<TH>::Warps;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const StyleView sv = StyleView::of(a);
    const VoteMasks<R, TH> mk = VoteMasks<R, TH>::at(smem + L.off_masks);
    uint32_t *const T = reinterpret_cast<uint32_t *>(smem + L.off_gt);
    int *const cnt = reinterpret_cast<int *>(smem + L.off_cnt);
    // the two pixel lists share one area: two-run windows from its start,
    // tap-by-tap windows downwards from entry 64 TH - 1 (the classes are
    // disjoint, so together they hold at most the tile's 64 TH pixels)
    uint16_t *const glist = reinterpret_cast<uint16_t *>(smem + L.off_lists);
    uint16_t *const tlist = glist + (kTW * TH - 1);
    const int wcols = min(a.W - x0, kTW);  // columns of the tile inside the target
    const uint64_t incols = wcols >= 64 ? ~0ull : ((1ull << wcols) - 1ull);
    if (R > 0 && threadIdx.x == 0) cnt[3] = cnt[4] = 0;  // two-runs and tap-by-tap list lengths

    if constexpr (R > 0) {
        // per region pixel: T = texel index of A (kNoTexel outside the
        // source); per region row: E bit x <=> A[x] == A[x-1] + 1, V bit x
        // <=> A[ry][x] == A[ry-1][x] + (0, 1) (never true next to kInvalid),
        // N bit x <=> A[x] lies at least R pixels inside the source, so every
        // tap it gives a window lies in the source
        const uint32_t iw = sv.Ws > 2u * R ? sv.Ws - 2u * R : 0u;
        const uint32_t ih16 = (sv.Hs16 >> 16) > 2u * R ? sv.Hs16 - (2u * R << 16) : 0u;
        // columns 0..63: a warp per row, 32 columns per ballot
        for (int ry = warp; ry < RH; ry += kWarps) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                bool eb, vb, nb;
                pixel_bits<R, RW, kTrustA>(A, T, sv, iw, ih16, ry, c * 32 + lane, eb, vb, nb);
                const uint32_t e = __ballot_sync(0xFFFFFFFFu, eb);
                const uint32_t v = __ballot_sync(0xFFFFFFFFu, vb);
                const uint32_t nn = __ballot_sync(0xFFFFFFFFu, nb);
                if (lane == 0) {
                    mk.E[4 * ry + c] = e;
                    mk.V[4 * ry + c] = v;
                    mk.N[4 * ry + c] = nn;
                }
            }
        }
        // columns 64..63+2R of 32 / 2R rows at once (lane = row * 2R + column)
        {
            constexpr int kCw = 2 * R, kRows = 32 / kCw, kIters = (RH + kRows - 1) / kRows;
            const int rl = lane / kCw, col = lane - rl * kCw;
            for (int it = warp; it < kIters; it += kWarps) {
                const int ry = it * kRows + rl;
                const bool valid = rl < kRows && ry < RH;
                bool eb = false, vb = false, nb = false;
                if (valid) pixel_bits<R, RW, kTrustA>(A, T, sv, iw, ih16, ry, 64 + col, eb, vb, nb);
                const uint32_t e = __ballot_sync(0xFFFFFFFFu, eb);
                const uint32_t v = __ballot_sync(0xFFFFFFFFu, vb);
                const uint32_t nn = __ballot_sync(0xFFFFFFFFu, nb);
                if (valid && col == 0) {
                    constexpr uint32_t kM = kCw >= 32 ? 0xFFFFFFFFu : (1u << kCw) - 1u;
                    const int sh = rl * kCw;
                    mk.E[4 * ry + 2] = (e >> sh) & kM;
                    mk.V[4 * ry + 2] = (v >> sh) & kM;
                    mk.N[4 * ry + 2] = (nn >> sh) & kM;
                    mk.E[4 * ry + 3] = mk.V[4 * ry + 3] = mk.N[4 * ry + 3] = 0u;
                }
            }
        }
        __syncthreads();
        // one thread per region row, 64 output columns at once: hu bit tx <=>
        // window row tx..tx+2R is one run; t2 <=> at most two runs; vc <=> the
        // centre column is linked to the row above; ni <=> every pixel of the
        // window row is interior
        if (threadIdx.x < RH) {
            const int ry = threadIdx.x;
            const uint32_t *e = mk.E + 4 * ry, *v = mk.V + 4 * ry, *nw = mk.N + 4 * ry;
            const uint64_t blo = ~((uint64_t)e[0] | ((uint64_t)e[1] << 32)), bhi = ~(uint64_t)e[2];
            const uint64_t ilo = (uint64_t)nw[0] | ((uint64_t)nw[1] << 32), ihi = nw[2];
            uint64_t seen = 0, two = 0, in = ilo;
            constexpr int kUnroll = R <= 7 ? 2 * R : 1;
#pragma unroll kUnroll
            for (int s = 1; s <= 2 * R; ++s) {
                const uint64_t b = shr128(blo, bhi, s);
                two |= seen & b;
                seen |= b;
                in &= shr128(ilo, ihi, s);
            }
            mk.hu[ry] = ~seen;
            mk.t2[ry] = ~two;
            mk.vc[ry] = shr128((uint64_t)v[0] | ((uint64_t)v[1] << 32), v[2], R);
            mk.ni[ry] = in;
        }
        __syncthreads();
        // four threads per output row, 16 columns each: the row's classes
        // (uniform windows; interior windows whose rows have at most two runs;
        // the rest, flagged when interior) and its entries of the two lists
        if (threadIdx.x < 4 * TH) {
            const int ty = threadIdx.x >> 2, sl = threadIdx.x & 3;
            uint64_t U = mk.hu[ty], T2 = mk.t2[ty], NI = mk.ni[ty];
#pragma unroll
            for (int k = 1; k <= 2 * R; ++k) {
                U &= mk.hu[ty + k] & mk.vc[ty + k];
                T2 &= mk.t2[ty + k];
                NI &= mk.ni[ty + k];
            }
            const uint64_t in = y0 + ty < a.H ? incols : 0ull;
            U &= in;
            const uint64_t G = T2 & NI & ~U & in, Tt = ~U & ~G & in;
            if (sl == 0) mk.U[ty] = U;
            uint32_t g16 = (uint32_t)(G >> (16 * sl)) & 0xFFFFu;
            uint32_t t16 = (uint32_t)(Tt >> (16 * sl)) & 0xFFFFu;
            const uint32_t n16 = (uint32_t)(NI >> (16 * sl));
            int ng, nt;
            int og = warp_exclusive_scan(__popc(g16), ng);
            int ot = warp_exclusive_scan(__popc(t16), nt);
            int bg = 0, bt = 0;
            if (lane == 0) {
                if (ng) bg = atomicAdd(&cnt[3], ng);
                if (nt) bt = atomicAdd(&cnt[4], nt);
            }
            og += __shfl_sync(0xFFFFFFFFu, bg, 0);
            ot += __shfl_sync(0xFFFFFFFFu, bt, 0);
            const int k0 = ty * kTW + 16 * sl;
            while (g16) {
                const int b = __ffs(g16) - 1;
                glist[og++] = (uint16_t)(k0 + b);
                g16 &= g16 - 1u;
            }
            while (t16) {
                const int b = __ffs(t16) - 1;
                tlist[-(ot++)] = (uint16_t)((k0 + b) | ((n16 >> b) & 1u ? kInteriorFlag : 0));
                t16 &= t16 - 1u;
            }
        }
        __syncthreads();
    }
    // output rows: warp w takes rows w, w + 8, ...  A uniform window votes
    // exactly C_S[A(p)] (all its taps share one source position; outside the
    // source the vote is 0); the other pixels are in the two lists.
    constexpr int kRowsPerWarp = TH / kWarps;
    uint32_t col[kRowsPerWarp][2];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
        const int ty = warp + q * kWarps;
        uint64_t U;
        if constexpr (R > 0) U = mk.U[ty];
        else U = y0 + ty < a.H ? incols : 0ull;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int tx = c * 32 + lane;
            col[q][c] = 0;
            if ((U >> tx) & 1ull) {
                if constexpr (R > 0) {
                    const uint32_t i = T[(ty + R) * RW + tx + R];
                    if (i != kNoTexel) col[q][c] = sv.texel(i);
                } else {
                    const uint32_t v = A[ty * RW + tx];
                    if (sv.in_source(v)) col[q][c] = sv.at(v);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
        const int ty = warp + q * kWarps;
        uint64_t U;
        if constexpr (R > 0) U = mk.U[ty];
        else U = y0 + ty < a.H ? incols : 0ull;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int tx = c * 32 + lane;
            if ((U >> tx) & 1ull) {
                if constexpr (F32) {
                    // outside the source col is 0, which votes (0, 0, 0, 0)
                    a.f32_out[(int64_t)(y0 + ty) * a.W + x0 + tx] = rgba_f32(col[q][c]);
                } else {
                    a.rgba_out[(int64_t)(y0 + ty) * a.W + x0 + tx] = col[q][c];
                }
            }
        }
    }
    if constexpr (R > 0) {
        vote_two_runs<R, F32, kThreads>(a, sv, T, mk.E, glist, cnt[3], x0, y0);
        vote_taps<R, F32, kThreads>(a, sv, A, T, tlist, cnt[4], x0, y0);
    }
}

// One 64 x TH output tile (tile_x, tile_y) of one frame.
template <int C, int B, int MODE, int R, int TH = kTH>
__device__ __forceinline__ void frame_tile(const FrameArgs &a, const SmemLayout &L, int tile_x,
                                           int tile_y, unsigned char *smem) {
    const int x0 = tile_x * kTW, y0 = tile_y * TH;
    uint8_t *bytes = smem + L.off_bytes;
    assign_region<C, B, R, TH>(a, L, x0 - R, y0 - R, smem, MODE == kAssign ? bytes : nullptr);
    const uint32_t *A = reinterpret_cast<const uint32_t *>(smem + L.off_A);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (MODE == kAssign) {
        for (int ty = warp; ty < TH; ty += Tile<TH>::Warps) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int tx = c * 32 + lane;
                const int gx = x0 + tx, gy = y0 + ty;
                if (gx < a.W && gy < a.H) {
                    a.assign_out[(int64_t)gy * a.W + gx] = A[ty * kTW + tx];
                    if (a.level_out) a.level_out[(int64_t)gy * a.W + gx] = bytes[ty * kTW + tx];
                }
            }
        }
    } else {
        vote_tile<R, false, TH>(a, L, x0, y0, A, smem);
    }
}

// CTAs per SM the kernels are compiled for: four (64 registers a thread) hide
// more of each tile's load latency than three with 80 registers; five (48)
// spill too much.  Windows above 15 x 15 need more than a quarter of the
// SM's shared memory anyway, so they are compiled for one CTA per SM.  Other
// tile heights keep 64 registers a thread: 8, 4 or 2 CTAs of 128, 256 or 512
// threads.
__host__ __device__ constexpr int min_ctas(int r, int th = kTH) { return r <= 7 ? 128 / th : 1; }

template <int C, int B, int MODE, int R>
__global__ void __launch_bounds__(Tile<kTH>::Threads, min_ctas(R))
    frame_kernel(const FrameArgs a, const SmemLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    frame_tile<C, B, MODE, R>(a, L, blockIdx.x, blockIdx.y, smem);
}

// Many frames in one launch: block b stylises tile b - tile_start[k] of the
// frame k with tile_start[k] <= b < tile_start[k + 1].  Frames may differ in
// size, exemplar, levels, threshold and seed; they share the guide format and
// the blend radius.  One launch lets the tiles of later frames fill the SMs
// while the last tiles of earlier frames finish.
constexpr int kMaxBatch = 128;

// floor(n / d) for 0 <= n < 2^31 and 1 <= d < 2^31 by one widening multiply:
// with l = ceil(log2 d) and m = ceil(2^(31 + l) / d), floor(n / d) =
// floor(n m / 2^(31 + l)) for every such n (Granlund and Montgomery, "Division
// by invariant integers using multiplication", PLDI 1994, Theorem 4.2: m d -
// 2^(31 + l) < d <= 2^l).  m has at most 33 bits, so n m fits 64 bits.
struct FastDiv {
    uint64_t m;
    uint32_t shift;  // 31 + l
    static FastDiv of(uint32_t d) {
        uint32_t l = 0;
        while ((1ull << l) < d) ++l;
        const uint32_t sh = 31 + l;
        return FastDiv{((1ull << sh) + d - 1) / d, sh};
    }
    __device__ __forceinline__ int operator()(int n) const {
        return (int)(((uint64_t)(uint32_t)n * m) >> shift);
    }
};

struct BatchArgs {
    int n;
    // tile order: 0 frame by frame; otherwise (every frame has rows_tx x
    // rows_ty tiles) tile row r of every frame before tile row r + 1, so the
    // exemplar lines those rows gather stay in L2 across the frames
    int rows_interleaved;
    int rows_tx;
    FastDiv div_row;      // by n * rows_tx, the tiles of one interleaved tile row
    FastDiv div_rows_tx;  // by rows_tx
    int tile_start[kMaxBatch + 1];
    int tiles_x[kMaxBatch];
    FastDiv div_tiles_x[kMaxBatch];
    FrameArgs f[kMaxBatch];
};

// Tile t of a batch: the frame k with tile_start[k] <= t < tile_start[k + 1]
// (frame by frame), or tile row t / (n * rows_tx) of frame (t / rows_tx) % n
// (rows interleaved).
template <int C, int B, int R, int TH>
__device__ __forceinline__ void batch_tile(const BatchArgs &b, const SmemLayout &L, int t,
                                           unsigned char *smem) {
    // the tile's frame k and position, then one inlined tile body for both
    // orders (two would double the kernel's code and its register pressure)
    int k, tx, ty;
    if (b.rows_interleaved) {
        ty = b.div_row(t);
        const int rem = t - ty * (b.n * b.rows_tx);
        k = b.div_rows_tx(rem);
        tx = rem - k * b.rows_tx;
    } else {
        int lo = 0, hi = b.n - 1;  // last frame whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.tile_start[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        k = lo;
        const int lt = t - b.tile_start[k];
        ty = b.div_tiles_x[k](lt);
        tx = lt - ty * b.tiles_x[k];
    }
    const FrameArgs a = b.f[k];  // register copy: field reads become plain operands
    frame_tile<C, B, kStylize, R, TH>(a, L, tx, ty, smem);
}

template <int C, int B, int R, int TH>
__global__ void __launch_bounds__(Tile<TH>::Threads, min_ctas(R, TH))
    batch_kernel(const __grid_constant__ BatchArgs b, const SmemLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    batch_tile<C, B, R, TH>(b, L, (int)blockIdx.x, smem);
}

// Work queue of a persistent batch launch: CTAs take the next tile from
// `next` until the batch is exhausted; the last CTA to leave clears the queue
// for the next launch that uses it (CUDA graph replays included).  The host
// hands every launch a queue no launch that may run at the same time holds
// (sb_frame_api.cu).  No CTA waits on another.
struct TileQueue {
    unsigned int next, done;
};

template <int C, int B, int R, int TH>
__global__ void __launch_bounds__(Tile<TH>::Threads, min_ctas(R, TH))
    batch_kernel_persistent(const __grid_constant__ BatchArgs b, const SmemLayout L,
                            TileQueue *q) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int tile;
    const int n_tiles = b.tile_start[b.n];
    for (;;) {
        if (threadIdx.x == 0) tile = (int)atomicAdd(&q->next, 1u);
        __syncthreads();
        const int t = tile;
        __syncthreads();  // every thread has read `tile` before it is overwritten
        if (t >= n_tiles) break;
        batch_tile<C, B, R, TH>(b, L, t, smem);
        __syncthreads();  // the tile's shared memory is free before the next tile writes it
    }
    if (threadIdx.x == 0) {
        // this CTA takes no more tiles; the last one out resets the queue
        if (atomicAdd(&q->done, 1u) == gridDim.x - 1) {
            atomicExch(&q->next, 0u);
            atomicExch(&q->done, 0u);
        }
    }
}

template <bool F32, int R>
__global__ void __launch_bounds__(Tile<kTH>::Threads) blend_kernel(const FrameArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int RW = kTW + 2 * R, NR = RW * (kTH + 2 * R);
    const SmemLayout L = smem_layout(R, 0);
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int rx0 = x0 - R, ry0 = y0 - R;
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
#pragma unroll 4
    for (int i = threadIdx.x; i < NR; i += Tile<kTH>::Threads) {
        const int gx = rx0 + i % RW, gy = ry0 + i / RW;
        const bool inside = gx >= 0 && gy >= 0 && gx < a.W && gy < a.H;
        A[i] = inside ? __ldg(a.assign_in + (int64_t)gy * a.W + gx) : kInvalid;
    }
    __syncthreads();
    vote_tile<R, F32, kTH, false>(a, L, x0, y0, A, smem);
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, device);
// later launches of no larger size skip the runtime call.  The cache is keyed
// by the kernel itself (one static per template instance).
template <auto Kernel>
cudaError_t ensure_smem(size_t smem) {
    constexpr int kMaxDev = 64;
    static std::atomic<uint32_t> done[kMaxDev] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t need = (uint32_t)smem;
    if (dev < kMaxDev && done[dev].load(std::memory_order_relaxed) >= need) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess && dev < kMaxDev) {
        uint32_t cur = done[dev].load();
        while (cur < need && !done[dev].compare_exchange_weak(cur, need)) {
        }
    }
    return e;
}

template <auto Kernel, typename... Args>
cudaError_t launch_tiles(size_t smem, int W, int H, cudaStream_t s, const Args &...args) {
    cudaError_t e = ensure_smem<Kernel>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    Kernel<<<grid, Tile<kTH>::Threads, smem, s>>>(args...);
    return cudaGetLastError();
}

template <int C, int B, int R>
cudaError_t launch_stylize_r(const FrameArgs &a, cudaStream_t s) {
    const SmemLayout L = smem_layout(R, a.levels);
    return launch_tiles<frame_kernel<C, B, kStylize, R>>(L.total, a.W, a.H, s, a, L);
}

// CTAs of a persistent launch: as many as fit on the device at once (cached
// per kernel, device and shared-memory size), at most one per tile.
template <auto Kernel>
int persistent_grid(size_t smem, int threads, int n_tiles) {
    constexpr int kMaxDev = 64;
    static std::atomic<uint64_t> cache[kMaxDev] = {};  // smem << 32 | CTAs
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t c = dev < kMaxDev ? cache[dev].load(std::memory_order_relaxed) : 0;
    int ctas = 0;
    if (c && (c >> 32) == smem) {
        ctas = (int)(c & 0xFFFFFFFFu);
    } else {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, threads, smem);
        ctas = max(1, sms * max(per_sm, 1));
        if (dev < kMaxDev) cache[dev].store(((uint64_t)smem << 32) | (uint32_t)ctas);
    }
    return min(ctas, n_tiles);
}

template <int C, int B, int R, int TH>
cudaError_t launch_batch_rt(const BatchArgs &b, int max_levels, TileQueue *queue, cudaStream_t s) {
    // one layout (for the deepest frame) serves every tile of the launch
    constexpr int kThreads = Tile<TH>::Threads;
    const SmemLayout L = smem_layout(R, max_levels, false, TH);
    const int n_tiles = b.tile_start[b.n];
    if (!queue) {
        cudaError_t e = ensure_smem<batch_kernel<C, B, R, TH>>(L.total);
        if (e != cudaSuccess) return e;
        batch_kernel<C, B, R, TH><<<n_tiles, kThreads, L.total, s>>>(b, L);
        return cudaGetLastError();
    }
    cudaError_t e = ensure_smem<batch_kernel_persistent<C, B, R, TH>>(L.total);
    if (e != cudaSuccess) return e;
    const int grid =
        persistent_grid<batch_kernel_persistent<C, B, R, TH>>(L.total, kThreads, n_tiles);
    batch_kernel_persistent<C, B, R, TH><<<grid, kThreads, L.total, s>>>(b, L, queue);
    return cudaGetLastError();
}

// Blend radii with tiles of 16 and 64 rows besides the default 32, and the
// largest radius of the first of the two radius ranges each format compiles in
// separate translation units (they compile in parallel).
constexpr int kMaxShapedRadius = 7;
constexpr int kNarrowMaxRadius = 7;

// Launches the batch kernel of guide format <C, B> for blend radius r in
// [R, RMax] with tiles of 32 rows (launch_batch32) or of th = 16 or 64 rows (r
// <= kMaxShapedRadius, launch_batch_shaped): one CTA per tile (queue ==
// nullptr) or persistent CTAs over the given work queue.
template <int C, int B, int R, int RMax>
cudaError_t launch_batch32(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                           cudaStream_t s) {
    if (r == R) return launch_batch_rt<C, B, R, 32>(b, max_levels, queue, s);
    if constexpr (R < RMax) return launch_batch32<C, B, R + 1, RMax>(b, r, max_levels, queue, s);
    return cudaErrorInvalidValue;
}

template <int C, int B, int R = 0>
cudaError_t launch_batch_shaped(const BatchArgs &b, int r, int th, int max_levels,
                                TileQueue *queue, cudaStream_t s) {
    if (r == R) {
        if (th == 16) return launch_batch_rt<C, B, R, 16>(b, max_levels, queue, s);
        if (th == 64) return launch_batch_rt<C, B, R, 64>(b, max_levels, queue, s);
        return cudaErrorInvalidValue;
    }
    if constexpr (R < kMaxShapedRadius)
        return launch_batch_shaped<C, B, R + 1>(b, r, th, max_levels, queue, s);
    return cudaErrorInvalidValue;
}

// The fused frame kernel for blend radius a.radius in [R, RMax].
template <int C, int B, int R, int RMax>
cudaError_t launch_stylize(const FrameArgs &a, cudaStream_t s) {
    if (a.radius == R) return launch_stylize_r<C, B, R>(a, s);
    if constexpr (R < RMax) return launch_stylize<C, B, R + 1, RMax>(a, s);
    return cudaErrorInvalidValue;
}

// Launches the frame kernel of guide format <C, B> in the given mode (the
// fused kernel for radii up to kNarrowMaxRadius; the wider ones through
// launch_frame_wide_c<C>b<B>).
template <int C, int B>
cudaError_t launch_frame_narrow(int mode, const FrameArgs &a, cudaStream_t s) {
    if (mode == kAssign) {
        const SmemLayout L = smem_layout(0, a.levels, true);
        return launch_tiles<frame_kernel<C, B, kAssign, 0>>(L.total, a.W, a.H, s, a, L);
    }
    return launch_stylize<C, B, 0, kNarrowMaxRadius>(a, s);
}

// per-format launchers: frame kernels and 32-row batches of radii up to 7 in
// sb_frame_c<C>b<B>.cu, radii 8-15 in sb_frame_c<C>b<B>_wide.cu, 16- and 64-row
// batches in sb_frame_c<C>b<B>_shapes.cu
cudaError_t launch_frame_c1b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c1b8(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c1b8(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c1b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c1b8(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);
cudaError_t launch_frame_c2b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c2b8(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c2b8(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c2b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c2b8(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);
cudaError_t launch_frame_c3b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c3b8(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c3b8(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c3b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c3b8(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);
cudaError_t launch_frame_c4b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c4b8(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c4b8(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c4b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c4b8(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);
cudaError_t launch_frame_c1b16(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c1b16(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c1b16(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c1b16(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c1b16(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);
cudaError_t launch_frame_c2b16(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_wide_c2b16(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_batch_c2b16(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s);
cudaError_t launch_batch_wide_c2b16(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s);
cudaError_t launch_batch_shaped_c2b16(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s);

}  // namespace sb
